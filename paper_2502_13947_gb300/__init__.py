"""GB300 (sm_103a) implementation of the data-parallel hot path of IC-D2S
(Abdollahi, Kamal, Pedram, ASP-DAC'25): Tabu search, control parameters,
subQUBO selection, the emulated Ising machine, exact gain write-back and
mutation, behind the C ABI in include/icd2s.h.

Submodules: ``icd2s`` (ctypes binding of libicd2s.so), ``build`` (nvcc build),
``instances`` (seeded synthetic QUBO instances), ``shard`` (one problem over
several GPUs: replica shards and their two collectives).  Importing the package does
not load the CUDA library; the first call into ``icd2s`` does, and raises if
it is missing.
"""
