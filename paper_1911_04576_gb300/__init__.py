"""GB300 (sm_103a) implementation of the FFT-accelerated macromodel lattice
solver of Patel, Triverio and Hum for inhomogeneous EM surfaces.

The compute path lives in ``libemsurf.so`` (CUDA, built by ``build.py``);
``binding`` marshals arguments to its C ABI (``include/emsurf.h``);
``workloads`` holds the seeded synthetic input recipes.
"""
