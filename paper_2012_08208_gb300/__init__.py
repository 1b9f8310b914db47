"""GB300-native hot path of the SIMP topology-optimisation loop of
arXiv 2012.08208: matrix-free K(rho)u (Q4 / H8) inside Jacobi-PCG, the
mesh-independency filter, element sensitivities and the OC bisection update,
as hand-written CUDA kernels behind a C-ABI (include/topo.h).

`paper_2012_08208_gb300.topo` is the ctypes binding; importing it requires the
built library (`paper_2012_08208_gb300/_lib/libtopo.so`).
"""
