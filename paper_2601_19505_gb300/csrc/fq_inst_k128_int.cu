// Kernels for 128-bit addresses with INT amplitudes (all Hamiltonian kinds).
#include "fq_launch.cuh"
FQ_INSTANTIATE(register_k128_int, fq::u128, FQ_AMP_INT)
