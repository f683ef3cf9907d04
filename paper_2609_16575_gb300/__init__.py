"""GB300-native hot path of the explicit electromagnetic PIC cycle of KEMPIC-3D
(arxiv 2609.16575): staggered CIC gather, relativistic Boris push, zigzag
charge-conserving current deposit and Yee FDTD updates, written as CUDA kernels
for sm_103a behind a C ABI (``include/gbpic.h``).

``paper_2609_16575_gb300.gbpic`` is the thin ctypes binding of that ABI; it
loads the in-tree ``libgbpic.so`` on first use and raises if it is missing.
``paper_2609_16575_gb300.workloads`` draws the seeded synthetic inputs.
"""
