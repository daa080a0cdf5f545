// Launchers of the adjoint through the scattering source iteration (the transpose of Alg. 1).
#pragma once
#include "common.cuh"

namespace sw {

// dL/dkappa_a, dL/deps accumulated over directions d0..d0+nd-1 (as launch_grad_accum), and, with
// J != nullptr, dL/dkappa_s = V sum_d lambda_d (J - I_d) written to gks.
cudaError_t launch_grad_scat(int precision, const void* I, const void* lam, int64_t N, int G, int nd, int d0,
                             const double* w64, const double* vol, const double* dl_dG, const double* J, double* gk,
                             double* ge, double* gks, cudaStream_t st);

// One step of the transposed source iteration: mu+- = sum_d lambda+-_d of the split adjoint sweep,
// d_max[0] = max |change of mu|, d_max[1] = max |mu| (both as FP64 bit patterns, atomically maxed:
// zero them first), and the split sources g+- + kappa_s V mu+- / 4pi of the next transposed sweep.
cudaError_t launch_adjoint_mu(int precision, const void* lam, int64_t N, int G, int nd, const double* vol,
                              const double* ka, const double* ks, const double* dl_dJ, const double* dl_dG,
                              double* mu, float2* cm32, double2* cm64, unsigned long long* d_max, cudaStream_t st);

}  // namespace sw
