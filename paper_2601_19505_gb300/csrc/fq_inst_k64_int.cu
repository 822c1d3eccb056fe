// Kernels for 64-bit addresses with INT amplitudes (all Hamiltonian kinds).
#include "fq_launch.cuh"
FQ_INSTANTIATE(register_k64_int, uint64_t, FQ_AMP_INT)
