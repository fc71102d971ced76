"""GB300-native Bezier Splatting rasterizer: CUDA kernels behind a C ABI.

``paper_2503_16424_gb300.bs`` is the thin ctypes binding of libbs.so (it
raises ImportError when the library has not been built);
``paper_2503_16424_gb300.synth`` makes seeded synthetic inputs.
"""
