"""GB300 (sm_103a) library for the dG spherical-harmonic Vlasov--Fokker--Planck operator of
arXiv:2501.05110: C ABI in include/sap.h, CUDA sources in csrc/, ctypes binding in sapgpu.py,
seeded synthetic workloads in workloads.py."""
