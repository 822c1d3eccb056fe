// Kernels for 128-bit addresses with F64 amplitudes (all Hamiltonian kinds).
#include "fq_launch.cuh"
FQ_INSTANTIATE(register_k128_f64, fq::u128, FQ_AMP_F64)
