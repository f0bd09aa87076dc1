"""GB300-native PRISM STEM simulation (Ophus 2017): compact S-matrix build, probe scan and the
per-probe multislice baseline as hand-written sm_103a CUDA kernels behind a C ABI (libprism.so).

Modules: ``prism`` (ctypes binding, same names as include/prism.h), ``runtime`` (torch-facing
wrapper), ``specimens`` (seeded synthetic inputs), ``build`` (nvcc build of the library).
Importing the package loads nothing; the library is loaded on first use and its absence raises.
"""
