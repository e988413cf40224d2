// Host view of the Navier-Stokes stage kernel (device code: ns.cu).
#pragma once
#include "args.h"

namespace fft3d {

// One Heun (RK2) stage on the velocity half-spectra, every array 3 fields of
// M = n0*n1*H complex values (6 for nhat), field stride M.
//   stage 1: ustar = u + dt R(u),  acc = u + dt/2 R(u)   (reads u, nhat = N(u))
//   stage 2: u = acc + dt/2 R(ustar)                     (reads ustar, nhat = N(ustar), acc)
// R = mask * (-i P(k) (k_j N_lj) - nu |k|^2 u).
struct NsArgs {
    float2* u;
    float2* ustar;
    float2* acc;
    const float2* nhat;
    int n0, n1, n2, H;
    long long M;
    float nu, dt;
};

cudaError_t launch_ns_stage(const NsArgs& a, int stage, cudaStream_t s);

}  // namespace fft3d
