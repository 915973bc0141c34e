"""GB300-native differentiable cloth simulator step and adjoint (phi-SfT, Sec. 3.1).

The compute path is the C-ABI CUDA library ``_lib/libcloth_sim.so`` (sources in
``csrc/``, header ``include/cloth_sim.h``); ``sim`` is its Python binding and
``workloads`` generates seeded synthetic inputs.
"""
__all__ = ["sim", "workloads", "build"]
