"""GB300-native time multigrid for DG-in-time discretisations (Gander & Neumueller, arXiv:1409.5254).

``tmg``        -- Python binding of the C ABI (include/tmg.h) over libtmg.so
``inputs``     -- seeded synthetic workloads
``build_ext``  -- nvcc build of libtmg.so for sm_103a
``autograd``   -- torch.autograd.Function over the batched solve and adjoint
``replicas``   -- host logic of multi-rank runs (replicas, instance shards, timing reduction)
The CUDA library is loaded lazily on first use so that the input generators
import on machines without a GPU.
"""
__all__ = ["tmg", "inputs", "build_ext", "autograd", "replicas"]
