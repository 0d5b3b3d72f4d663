// Projector values formed where they are used (no N_p x npw table): for
// projector p = a nproj + c at plane wave g, q = k + G,
//     beta_p(q) = f_c(|q|) (1 or -i) e^{-i q_x X_a} e^{-i q_y Y_a} e^{-i q_z Z_a},
// with f_c the real radial factor of type c (times sqrt(2) w q_axis for p
// types) stored per plane wave, and the phase as the product of three
// per-atom one-axis tables (the cell is orthorhombic, so e^{-i q.R} factorises).
#pragma once

#include "fs_common.cuh"

struct BetaGen {
    const double* rad;    // [nproj][npw] radial factor f_c
    const double2* ph;    // [natom][3][span] e^{-i q_d R_{a,d}} for g_d = lo_d + j
    const float* rad32;   // the same tables rounded to FP32 (the FP32 stage's operand images)
    const float2* ph32;
    const int* gidx;      // [npw] packed (j0 | j1 << 10 | j2 << 20)
    const int* pl;        // [nproj] 0 = s (factor 1), 1 = p (factor -i)
    int nproj, span;
    long npw;
};

__device__ __forceinline__ double2 beta_value(const BetaGen& B, int p, long g) {
    const int a = p / B.nproj, c = p - a * B.nproj;
    const double r = B.rad[(long)c * B.npw + g];
    const int code = B.gidx[g];
    const double2* ph = B.ph + (long)a * 3 * B.span;
    const double2 p0 = ph[code & 1023], p1 = ph[B.span + ((code >> 10) & 1023)],
                  p2 = ph[2 * B.span + ((code >> 20) & 1023)];
    const double2 e = cmul(cmul(p0, p1), p2);
    return B.pl[c] == 0 ? make_double2(r * e.x, r * e.y) : make_double2(r * e.y, -r * e.x);
}

// FP32 form for the FP32 stage's operand images (a few FP32 roundings, below the
// stage's own noise; FP64 arithmetic runs at a small fraction of the FP32 rate)
__device__ __forceinline__ float2 beta_value32(const BetaGen& B, int p, long g) {
    const int a = p / B.nproj, c = p - a * B.nproj;
    const float r = B.rad32[(long)c * B.npw + g];
    const int code = B.gidx[g];
    const float2* ph = B.ph32 + (long)a * 3 * B.span;
    const float2 e = cmul(cmul(ph[code & 1023], ph[B.span + ((code >> 10) & 1023)]), ph[2 * B.span + ((code >> 20) & 1023)]);
    return B.pl[c] == 0 ? make_float2(r * e.x, r * e.y) : make_float2(r * e.y, -r * e.x);
}

BetaGen beta_gen_of(const fs_ctx* c);
