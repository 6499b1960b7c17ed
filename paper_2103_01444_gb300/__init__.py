"""GB300-native coupled lattice-Boltzmann step for a PEM fuel-cell cathode
(arXiv 2103.01444): D2Q9 MRT flow with Darcy-Forchheimer drag, three D2Q5
MRT advection-diffusion fields (T, O2, H2O) and the catalyst-layer Tafel
reaction with its heat, as hand-written CUDA for sm_103a behind a C ABI.

Submodules are imported on demand: ``workloads`` (seeded inputs) needs
neither CUDA nor the compiled library.
"""
__all__ = ["workloads", "units", "lbm"]
