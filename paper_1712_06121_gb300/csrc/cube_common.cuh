// Shared device/host definitions of libcube's kernels (sm_103a).
//
// Geometry of the compressed store (Sections 2.1, 2.3.1 of the paper):
//   N  fine cells per side, Nc = N / R coarse cells per side,
//   coarse cells grouped in bricks of B^3 (brick-major storage order, cells
//   x-fastest inside a brick, bricks x-fastest), nb = Nc / B bricks per side.
// A particle in coarse cell c with code chi has, per dimension,
//   b = chi + 2^(8n-1) in [0, 2^(8n)),   Q = 2b + 1,
//   offset inside the cell = Q / 2^(8n+1) coarse cells      (Eq. x),
//   fine cell inside the coarse cell = Q >> s,  CIC weight = (Q & (2^s-1)) / 2^s,
//   with s = 8n + 1 - log2(R).  All of these are exact in FP32.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cube {

enum ErrFlag : uint32_t {
    ERR_MIGRATION = 1u,   // a particle moved more than one coarse cell
    ERR_NONFINITE = 2u,   // non-finite input position / velocity
    ERR_COUNT = 4u,       // counter overflow / inconsistent totals
};

struct Geo {
    int N;        // fine cells per side
    int Nc;       // coarse cells per side
    int R, r;     // fine cells per coarse cell, log2(R)
    int B;        // brick side (coarse cells)
    int nb;       // bricks per side
    int Bh;       // B + 2: brick plus one-cell halo on each side
    int nchi, nnu;
    int sbits;    // 8 nchi + 1 - r: bits of a CIC weight numerator
    int F;        // B * R: fine cells per brick side
    int S;        // mesh row stride in floats (N + 4)
    int Ncc;      // Nc^3
    int nbricks;  // nb^3
    int64_t Np;
    int nulim;    // 2^(8 nnu - 1) - 1: largest |nu|
};

// storage rank of coarse cell (cx, cy, cz), coordinates already in [0, Nc)
__host__ __device__ __forceinline__ int cell_rank(const Geo& g, int cx, int cy, int cz) {
    int bx = cx / g.B, by = cy / g.B, bz = cz / g.B;
    int lx = cx - bx * g.B, ly = cy - by * g.B, lz = cz - bz * g.B;
    return (bx + g.nb * (by + g.nb * bz)) * (g.B * g.B * g.B) + lx + g.B * (ly + g.B * lz);
}

__host__ __device__ __forceinline__ int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// 2^-24 fixed point of a velocity (round to nearest even); exact for |v| < 2^39
__device__ __forceinline__ long long vel_fix(float v) {
    return __float2ll_rn(v * 16777216.0f);
}

// v_c = mean of the cell's fixed-point velocities, rounded to FP32
__device__ __forceinline__ float vel_unfix_mean(long long s, unsigned n) {
    if (n == 0) return 0.0f;
    double m = __ll2double_rn(s) / (double)n;
    return __double2float_rn(m * (1.0 / 16777216.0));
}

// Eq. nu via exact thresholds: thr[k] (k = 1..lim) is the smallest float >=
// tan(pi (k - 1/2) / M) / s, thr[lim + 1] = +inf, so |d| >= thr[k]  <=>  the
// nearest integer of (M/pi) atan(|d| s) is >= k (halves away from zero).
// `est` is any starting guess; the result does not depend on it.
__device__ __forceinline__ int nu_from_thresholds(float d, const float* __restrict__ thr, int lim, int est) {
    float a = fabsf(d);
    int k = min(max(est, 0), lim);
    while (k < lim && a >= thr[k + 1]) ++k;
    while (k > 0 && a < thr[k]) --k;
    return d < 0.0f ? -k : k;
}

__device__ __forceinline__ int nu_estimate(float d, float m_over_pi_s, float m_over_pi) {
    return __float2int_rn(m_over_pi * atanf(fabsf(d) * m_over_pi_s));
}

template <int NB>
__device__ __forceinline__ int load_code(const void* base, int64_t idx) {
    if (NB == 1) return (int)reinterpret_cast<const int8_t*>(base)[idx];
    return (int)reinterpret_cast<const int16_t*>(base)[idx];
}

// velocity code clamped to the table range [-lim, lim] (the encoder never
// writes anything else; the clamp keeps table reads in bounds regardless)
template <int NB>
__device__ __forceinline__ int load_nu(const void* base, int64_t idx, int lim) {
    return max(-lim, min(lim, load_code<NB>(base, idx)));
}

template <int NB>
__device__ __forceinline__ void store_code(void* base, int64_t idx, int v) {
    if (NB == 1) reinterpret_cast<int8_t*>(base)[idx] = (int8_t)v;
    else reinterpret_cast<int16_t*>(base)[idx] = (int16_t)v;
}

// Drift inside the old coarse cell, identical in both re-sort passes:
// u_new = Q / 2^(8n+1) + p * dc  (one fused rounding).  Returns the bin
// floor(u_new * 2^(8n)) relative to the old cell's origin.
__device__ __forceinline__ int drift_bin(int Q, float p, float dc, float inv2q, float two8n, float* u_out) {
    float u = (float)Q * inv2q;
    float un = __fmaf_rn(p, dc, u);
    *u_out = un;
    return (int)floorf(un * two8n);
}

}  // namespace cube
