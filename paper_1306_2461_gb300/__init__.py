"""GB300-native dense pyramidal Lucas-Kanade optical flow (arXiv:1306.2461, Sect. 2.4).

The compute path is the CUDA library `libof.so` (sm_103a) behind a C ABI declared in
`include/of.h`; `paper_1306_2461_gb300.of` is its ctypes binding. `synth` generates
seeded synthetic particle-image workloads.
"""
