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
    ERR_TIMEOUT = 8u,     // a bounded wait for an asynchronous copy gave up
};

// Ghosted copy of the potential, written by the c2r sweep: x in [-4, N + 4),
// y and z in [-2, N + 3), values periodic, row stride N + 8 floats (a
// multiple of 16 bytes), so the Phi tile of any brick is one rectangular box.
constexpr int PHIG_X0 = 4, PHIG_Y0 = 2;
__host__ __device__ __forceinline__ int phig_nx(int N) { return N + 8; }
__host__ __device__ __forceinline__ int phig_ny(int N) { return N + 5; }
__host__ __device__ __forceinline__ int64_t phig_index(int N, int x, int y, int z) {
    return ((int64_t)(z + PHIG_Y0) * phig_ny(N) + (y + PHIG_Y0)) * phig_nx(N) + (x + PHIG_X0);
}

// ---- mbarrier and TMA (cp.async.bulk.tensor) wrappers
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// one potentially blocking test: the thread is suspended until the phase
// completes or about `hint_ns` nanoseconds pass (the hardware may wake it
// earlier); true if the phase completed
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity, unsigned hint_ns) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}
// waits at most 256 suspensions of up to 0.1 ms each (tens of milliseconds in
// all); false if the phase never completed.  A suspended thread issues no
// instructions, so waiting warps leave the issue slots to the SM's others.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    for (int it = 0; it < 256; ++it)
        if (mbar_try_wait(bar, parity, 100000u)) return true;
    return false;
}
// 3-D tiled TMA load of the tensor map's box at (x, y, z) into shared memory,
// completing on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// 4-D tiled TMA load (x, y, z, member) of the tensor map's box, completing on `bar`
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int x, int y, int z, int w,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
        : "memory");
}

// floor(t / d) for 0 <= t < 4096 and 2 <= d <= 8 as (t * ceil(2^16 / d)) >> 16
// (checked exhaustively over that range); m = div_magic(d)
__host__ __device__ __forceinline__ unsigned div_magic(int d) { return (65536u + (unsigned)d - 1u) / (unsigned)d; }
__host__ __device__ __forceinline__ int div_small(int t, unsigned m) { return (int)(((unsigned)t * m) >> 16); }

// the three coordinates of t = e0 + d (e1 + d e2), 0 <= t < d^3 <= 512
__device__ __forceinline__ void split3(int t, int d, unsigned m, int* e) {
    const int q = div_small(t, m);
    e[0] = t - q * d;
    e[2] = div_small(q, m);
    e[1] = q - e[2] * d;
}

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
    int nid;      // bytes per particle ID (n_I: 0, 1, 2 or 4)
    int lB, lF;   // log2(B), log2(F): brick and fine-tile sides are powers of two
    int nsm;      // SMs of the device (grid sizing)
};

// storage rank of coarse cell (cx, cy, cz), coordinates already in [0, Nc)
// (brick side B = 2^lB)
__host__ __device__ __forceinline__ int cell_rank(const Geo& g, int cx, int cy, int cz) {
    const int m = g.B - 1;
    const int bx = cx >> g.lB, by = cy >> g.lB, bz = cz >> g.lB;
    return ((bx + g.nb * (by + g.nb * bz)) << (3 * g.lB)) + (cx & m) + ((cy & m) << g.lB) + ((cz & m) << (2 * g.lB));
}

__host__ __device__ __forceinline__ int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// periodic wrap of a coordinate known to lie in [-n, 2n)
__host__ __device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Exact FP32 value of a 16-bit unsigned integer: 2^23 + u is a float, and
// subtracting 2^23 is exact.
__device__ __forceinline__ float u16_to_float(unsigned u) { return __int_as_float(0x4B000000 | u) - 8388608.0f; }

// Nearest FP32 to a 32-bit unsigned integer, from FP32 arithmetic alone:
// hi 2^16 + lo is formed exactly inside one fused multiply-add and rounded
// once.  (The integer-to-float conversion instructions issue at the FP64
// rate on this part.)
__device__ __forceinline__ float u32_to_float_rn(unsigned u) {
    return __fmaf_rn(u16_to_float(u >> 16), 65536.0f, u16_to_float(u & 0xffffu));
}

// 2^-24 fixed point of a velocity (round to nearest even); exact for |v| < 2^39
__device__ __forceinline__ long long vel_fix(float v) {
    return __float2ll_rn(v * 16777216.0f);
}

// v_c = mean of the cell's fixed-point velocities s / n, as the FP32 value
// fl32(fl64(s) / n * 2^-24).  For |s| < 2^53 and n < 2^27 the quotient s / n
// is either an FP32 rounding midpoint or at least 2^-52 (relative) away from
// every one -- more than FP64's half ulp -- so the FP64 rounding never moves
// the FP32 result: it is the correctly rounded fl32(s / n * 2^-24), formed
// here from a 64-bit integer quotient of 26-27 bits and a sticky bit (the
// FP64 division is very slow on this part).  Larger inputs divide in FP64.
__device__ __forceinline__ float vel_unfix_mean(long long s, unsigned n) {
    if (n == 0 || s == 0) return 0.0f;
    const unsigned long long a = s < 0 ? 0ull - (unsigned long long)s : (unsigned long long)s;
    if (a >= (1ull << 53) || n >= (1u << 27)) {
        const double m = __ll2double_rn(s) / (double)n;
        return __double2float_rn(m * (1.0 / 16777216.0));
    }
    const int la = 63 - __clzll((long long)a), ln = 31 - __clz((int)n);
    const int k = 26 - (la - ln);                      // shift giving a quotient in [2^25, 2^27)
    unsigned long long q;
    bool sticky;
    int e;
    if (k >= 0) {
        const unsigned long long num = a << k;         // < 2^53
        q = num / n;
        sticky = num - q * n != 0;
        e = -k;
    } else {
        q = a / n;
        sticky = a - q * n != 0;
        e = 0;
    }
    const int t = 64 - __clzll((long long)q) - 24;     // bits below the 24 kept
    const unsigned long long low = q & ((1ull << t) - 1), half = 1ull << (t - 1);
    unsigned long long q24 = q >> t;
    if (low > half || (low == half && (sticky || (q24 & 1)))) ++q24;   // nearest, ties to even
    const float v = ldexpf((float)q24, e + t - 24);
    return s < 0 ? -v : v;
}

// Eq. nu via exact thresholds: thr[k] (k = 1..lim) is the smallest float >=
// tan(pi (k - 1/2) / M) / s, thr[lim + 1] = +inf, so |d| >= thr[k]  <=>  the
// nearest integer of (M/pi) atan(|d| s) is >= k (halves away from zero).
// `est` is any starting guess; the result does not depend on it.
// The two thresholds around the guess are requested together, so a guess
// within one code costs one memory round trip.
__device__ __forceinline__ int nu_from_thresholds(float d, const float* __restrict__ thr, int lim, int est) {
    float a = fabsf(d);
    int k = min(max(est, 0), lim);
    const float lo = thr[k], hi = thr[k + 1];            // thr[lim + 1] = +inf
    if (a >= hi) {
        ++k;
        while (k < lim && a >= thr[k + 1]) ++k;
    } else if (a < lo) {
        --k;
        while (k > 0 && a < thr[k]) --k;
    }
    return d < 0.0f ? -k : k;
}

// Eq. nu for 1-byte codes through a bucket table.  Bucket i holds the |d|
// whose float bit patterns share bits 31..(23 - VT_B) = key0 + i: 2^VT_B
// buckets per octave, VT_N buckets (16 octaves) from just below thr[1].
// vtab[i] is the code of the bucket's first value.  Consecutive thresholds
// of 1-byte codes are at least 2.49% apart (relative; min over k of
// tan(pi (k + 1/2) / 255) / tan(pi (k - 1/2) / 255)), more than a bucket's
// width (at most 2^-6 = 1.56%), so a bucket holds at most one threshold and
// one compare with the next threshold completes the code; thr[1 .. 127]
// span 13.7 octaves, inside the table.  The result equals
// nu_from_thresholds'.
constexpr int VT_B = 6;
constexpr int VT_N = 1024;
__device__ __forceinline__ int nu_from_table(float d, const float* __restrict__ thr,
                                             const unsigned char* __restrict__ vtab, int key0, int lim) {
    const float a = fabsf(d);
    const int i = min(max((int)(__float_as_uint(a) >> (23 - VT_B)) - key0, 0), VT_N - 1);
    int k = vtab[i];
    k = min(k + (a >= thr[k + 1] ? 1 : 0), lim);
    return d < 0.0f ? -k : k;
}

// ---- 2-byte velocity tables as an approximation plus a 4-bit correction
// The decode values dec[k] = tan(pi k / M) gamma and the thresholds thr[k]
// (tan(pi (k - 1/2) / M) / s rounded up) of 2-byte codes are 2^16-entry
// tables whose entries a kernel reads at random: in global memory every
// lookup is an L2 round trip.  Both are tan(m pi / (2M)) gamma at m = 2k and
// m = 2k - 1, so each entry is stored as the difference, in ulps, between
// its exact FP32 value and tan_half_steps(m), a fixed FP32 evaluation that
// every kernel repeats bit for bit: 4 bits per entry (one byte holds both
// tables' corrections for one k), 32 KB that stay in L1.  A difference
// outside [-7, 7] is stored as -8 and that entry is read from the full table.
// The result is the table's value in every case; the approximation's
// accuracy only decides how rarely the full table is read.
struct VelApprox {
    float c;      // pi / (2M), M = 2 lim + 1
    float gam;    // sqrt(2 sigma^2 / pi) = 1 / s
    int M;
};

// tan(m pi / (2M)) gamma for 0 < m < M in FP32 to a few ulps: the angle, or
// above pi/4 its complement (M - m) pi / (2M) (tan = 1 / tan of the
// complement), lies in (0, pi/4], where the Taylor series of tan to x^23
// (Abramowitz & Stegun 4.3.67, coefficients 2^2n (2^2n - 1) |B_2n| / (2n)!)
// is within 5e-8 relative.  Explicitly rounded operations only, so every
// kernel gets the same bits.
__device__ __forceinline__ float tan_half_steps(int m, const VelApprox& va) {
    const bool cot = 2 * m > va.M;
    const int mm = cot ? va.M - m : m;                         // < 2^16
    const float x = __fmul_rn(__fsub_rn(__int_as_float(0x4B000000 | mm), 8388608.0f), va.c);
    const float x2 = __fmul_rn(x, x);
    float p = 3.9278322e-05f;
    p = __fmaf_rn(p, x2, 9.691538e-05f);
    p = __fmaf_rn(p, x2, 0.00023912912f);
    p = __fmaf_rn(p, x2, 0.0005900274f);
    p = __fmaf_rn(p, x2, 0.0014558344f);
    p = __fmaf_rn(p, x2, 0.003592128f);
    p = __fmaf_rn(p, x2, 0.008863236f);
    p = __fmaf_rn(p, x2, 0.021869488f);
    p = __fmaf_rn(p, x2, 0.053968254f);
    p = __fmaf_rn(p, x2, 0.13333334f);
    p = __fmaf_rn(p, x2, 0.33333334f);
    p = __fmaf_rn(p, x2, 1.0f);
    const float t = __fmul_rn(x, p);
    return cot ? __fdividef(va.gam, t) : __fmul_rn(t, va.gam);
}

// the signed 4-bit correction in bits lo..lo+3 of b
__device__ __forceinline__ int vdelta(unsigned b, int lo) { return (int)(b << (28 - lo)) >> 28; }

// the correction byte of k: decode difference in bits 0-3, threshold difference in bits 4-7
__device__ __forceinline__ unsigned char vdelta_pack(int dd, int dt) {
    const int a = (dd < -7 || dd > 7) ? -8 : dd, b = (dt < -7 || dt > 7) ? -8 : dt;
    return (unsigned char)((a & 15) | ((b & 15) << 4));
}

// exact 2-byte tables through the corrections; dec_g / thr_g the full tables
// (dec_g indexed by nu + lim), vdel [lim + 2] the correction bytes
struct VelTables {
    const float* __restrict__ dec_g;
    const float* __restrict__ thr_g;
    const unsigned char* __restrict__ vdel;
    VelApprox va;
    int lim;
    // dec[nu + lim] for |nu| <= lim
    __device__ __forceinline__ float dec(int nu) const {
        const int k = abs(nu);
        if (k == 0) return 0.0f;
        const int dd = vdelta(__ldg(&vdel[k]), 0);
        const float v = dd == -8 ? dec_g[k + lim]
                                 : __int_as_float(__float_as_int(tan_half_steps(2 * k, va)) + dd);
        return nu < 0 ? -v : v;
    }
    // thr[k] for 0 <= k <= lim + 1 (thr[0] = 0, thr[lim + 1] = +inf)
    __device__ __forceinline__ float thr(int k) const {
        if (k <= 0) return 0.0f;
        if (k > lim) return __int_as_float(0x7f800000);
        const int dt = vdelta(__ldg(&vdel[k]), 4);
        return dt == -8 ? thr_g[k] : __int_as_float(__float_as_int(tan_half_steps(2 * k - 1, va)) + dt);
    }
};

// nu_from_thresholds with the thresholds of a VelTables
__device__ __forceinline__ int nu_from_tables(float d, const VelTables& vt, int est) {
    const float a = fabsf(d);
    int k = min(max(est, 0), vt.lim);
    const float lo = vt.thr(k), hi = vt.thr(k + 1);
    if (a >= hi) {
        ++k;
        while (k < vt.lim && a >= vt.thr(k + 1)) ++k;
    } else if (a < lo) {
        --k;
        while (k > 0 && a < vt.thr(k)) --k;
    }
    return d < 0.0f ? -k : k;
}

// Starting guess for nu_from_thresholds: (M/pi) atan(|d| s) with the
// arctangent from the polynomial of Abramowitz & Stegun 4.4.47 (Hastings),
// |error| <= 1e-5 rad on [0, 1], and atan(x) = pi/2 - atan(1/x) above 1.
// The error is well under one code for 2-byte codes, so the exact search
// that follows takes at most a step or two.
__device__ __forceinline__ int nu_estimate(float d, float s, float m_over_pi) {
    const float x = fabsf(d) * s;
    const bool big = x > 1.0f;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));    // a guess needs no exact reciprocal
    const float t = big ? r : x;
    const float t2 = t * t;
    float p = 0.0208351f;
    p = __fmaf_rn(p, t2, -0.0851330f);
    p = __fmaf_rn(p, t2, 0.1801410f);
    p = __fmaf_rn(p, t2, -0.3302995f);
    p = __fmaf_rn(p, t2, 0.9998660f);
    float a = p * t;
    if (big) a = 1.57079633f - a;
    return __float2int_rn(m_over_pi * a);
}

// Packed FP32 pairs (Blackwell's two-wide FP32 instructions): each lane of a
// pair is rounded exactly as the scalar operation would round it.
__device__ __forceinline__ float2 pk2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n sub.rn.f32x2 z, x, y;\n"
        " mov.b64 {%0, %1}, z;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// 4th-order central differences 8 (f[1] - f[-1]) - (f[2] - f[-2]) at nodes 0
// and 1 of a line of six values f[-2 .. 3], for two lines at once, combined
// with the CIC weights w0 (node 0) and w1 (node 1)
__device__ __forceinline__ float2 fd4_cic_pair(const float2* r, float w0, float w1) {
    const float2 e8 = pk2(8.0f);
    const float2 g0 = pfma(e8, psub(r[3], r[1]), psub(r[0], r[4]));
    const float2 g1 = pfma(e8, psub(r[4], r[2]), psub(r[1], r[5]));
    return pfma(pk2(w1), g1, pmul(pk2(w0), g0));
}

// particle ID i of an n-byte ID array (n = 1, 2 or 4), zero-extended
__device__ __forceinline__ unsigned load_pid(const void* p, unsigned i, int n) {
    return n == 1 ? (unsigned)reinterpret_cast<const uint8_t*>(p)[i]
                  : n == 2 ? (unsigned)reinterpret_cast<const uint16_t*>(p)[i] : reinterpret_cast<const unsigned*>(p)[i];
}
// store the low n bytes of v as particle ID i
__device__ __forceinline__ void store_pid(void* p, unsigned i, int n, unsigned v) {
    if (n == 1) reinterpret_cast<uint8_t*>(p)[i] = (uint8_t)v;
    else if (n == 2) reinterpret_cast<uint16_t*>(p)[i] = (uint16_t)v;
    else reinterpret_cast<unsigned*>(p)[i] = v;
}

template <int NB> struct CodeType { using T = int8_t; };
template <> struct CodeType<2> { using T = int16_t; };

// The three axis rows of a [3][Np] code array as separate pointers, so a
// particle's codes are addressed by its 32-bit index alone.
template <int NB>
struct CodeRows {
    using T = typename CodeType<NB>::T;
    T* r[3];
    __device__ __forceinline__ CodeRows(const void* base, int64_t np) {
        r[0] = reinterpret_cast<T*>(const_cast<void*>(base));
        r[1] = r[0] + np;
        r[2] = r[1] + np;
    }
    __device__ __forceinline__ int get(int d, unsigned i) const { return (int)r[d][i]; }
    // velocity code clamped to [-lim, lim] (the encoder never writes anything
    // else; the clamp keeps table reads in bounds regardless)
    __device__ __forceinline__ int get_nu(int d, unsigned i, int lim) const { return max(-lim, min(lim, (int)r[d][i])); }
    __device__ __forceinline__ void put(int d, unsigned i, int v) const { r[d][i] = (T)v; }
};

template <int NB>
__device__ __forceinline__ int load_code(const void* base, int64_t idx) {
    if (NB == 1) return (int)reinterpret_cast<const int8_t*>(base)[idx];
    return (int)reinterpret_cast<const int16_t*>(base)[idx];
}

// ---- flattened (cell-major, brick-minor) order of the per-brick histograms
// A brick b sees the cells of its one-cell halo region, local index e in
// [0, Bh^3).  A coarse cell c lies in the regions of n_x n_y n_z bricks
// (per axis: its home brick, plus the lower neighbour if it is the first
// cell of the brick, plus the upper one if it is the last).  Ordering the
// (cell, brick) pairs by cell storage rank, then brick storage rank, gives a
// permutation of the nbricks * Bh^3 (brick, e) pairs; an exclusive scan in
// that order yields, for each pair, where brick b's particles moving into
// cell c start (stable by old index, since bricks are in storage order).

// candidates per axis for a cell at brick-local coordinate l
__host__ __device__ __forceinline__ int ncand(int l, int B) { return 1 + (l == 0) + (l == B - 1); }
// number of candidate slots of the cells before local coordinate l on an axis
__host__ __device__ __forceinline__ int ncand_before(int l) { return l + (l > 0); }

// first flattened slot of the cell with home brick hb (storage rank) and
// brick-local coordinates l[3]
__host__ __device__ __forceinline__ int64_t flat_base(const Geo& g, int hb, const int* l) {
    const int S1 = g.B + 2, S2 = S1 * S1;
    const int pre = ncand_before(l[2]) * S2 + ncand(l[2], g.B) * (ncand_before(l[1]) * S1 + ncand(l[1], g.B) * ncand_before(l[0]));
    return (int64_t)hb * (S2 * S1) + pre;
}

// flattened slot of (brick with coordinates bc[3], halo-region index e[3])
__host__ __device__ __forceinline__ int64_t flat_slot(const Geo& g, const int* bc, const int* e) {
    int l[3], hbc[3], rank = 0;
#pragma unroll
    for (int d = 2; d >= 0; --d) {
        const int c = wrap1((bc[d] << g.lB) - 1 + e[d], g.Nc);
        l[d] = c & (g.B - 1);
        hbc[d] = c >> g.lB;
        // candidate brick coordinates on this axis, ranked by value
        const int lo = (l[d] == 0) ? wrap1(hbc[d] - 1, g.nb) : -1;
        const int hi = (l[d] == g.B - 1) ? wrap1(hbc[d] + 1, g.nb) : -1;
        const int me = bc[d];
        int r = (hbc[d] < me) + (lo >= 0 && lo < me) + (hi >= 0 && hi < me);
        rank = rank * ncand(l[d], g.B) + r;
    }
    const int hb = hbc[0] + g.nb * (hbc[1] + g.nb * hbc[2]);
    return flat_base(g, hb, l) + rank;
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

// Asynchronous global -> shared copies (cp.async): all copies of a tile are
// issued before any is waited for, so the tile's load latency is paid once.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most one committed group (the most recent) is still in flight
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Lanes of `active` whose 8-bit value v (0 <= v < 256) equals this lane's:
// one ballot per bit, intersected.  Every lane of `active` must call it.
__device__ __forceinline__ unsigned same_value_lanes(unsigned active, int v) {
    unsigned m = active;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const unsigned bb = __ballot_sync(active, (v >> b) & 1);
        m &= ((v >> b) & 1) ? bb : ~bb;
    }
    return m;
}

// 64-bit add into shared memory from 32-bit atomics: the low word's
// wrap-arounds are carried into the high word, so the final value is the
// exact sum mod 2^64 whatever the order.  lohi = {low word, high word}.
// The block's largest v into *dst with one atomic (every thread of the block
// calls it; blockDim.x a multiple of 32).
__device__ __forceinline__ void block_max_to(unsigned v, unsigned* dst) {
    __shared__ unsigned wmax[32];
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned m = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0u;
        m = __reduce_max_sync(0xffffffffu, m);
        if (threadIdx.x == 0 && m) atomicMax(dst, m);
    }
}

// The block's sum of v into *dst with one atomic (integer: exact in any order)
__device__ __forceinline__ void block_sum_to(long long v, long long* dst) {
    __shared__ long long wsum[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += wsum[i];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)t);
    }
    __syncthreads();
}

__device__ __forceinline__ void smem_add_u64(unsigned* lohi, unsigned long long u) {
    const unsigned lo = (unsigned)u, hi = (unsigned)(u >> 32);
    const unsigned old = atomicAdd(&lohi[0], lo);
    const unsigned up = hi + ((old + lo < old) ? 1u : 0u);
    if (up) atomicAdd(&lohi[1], up);
}

// Drift inside the old coarse cell, identical in both re-sort passes:
// u_new = Q / 2^(8n+1) + p * dc (one fused rounding), formed in units of the
// position code's bins as x = Q / 2 + p * dcs = u_new 2^(8n), dcs = dc 2^(8n):
// scaling by a power of two commutes with the rounding, since no term is
// subnormal (a nonzero sum of Q / 2^(8n+1) and the 48-bit product p dc is at
// least 2^-64).  Q / 2 comes exactly from the bits of 2^22 + Q / 2 (Q < 2^23).
// Returns the bin floor(x) relative to the old cell's origin; *x_out = x.
__device__ __forceinline__ int drift_bin(int Q, float p, float dcs, float* x_out) {
    const float u0s = __int_as_float(0x4A800000 | Q) - 4194304.0f;
    const float x = __fmaf_rn(p, dcs, u0s);
    *x_out = x;
    return __float2int_rd(x);
}

}  // namespace cube
