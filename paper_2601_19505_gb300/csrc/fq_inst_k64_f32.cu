// Kernels for 64-bit addresses with F32 amplitudes (all Hamiltonian kinds).
#include "fq_launch.cuh"
FQ_INSTANTIATE(register_k64_f32, uint64_t, FQ_AMP_F32)
