// 3-D real FFT Poisson solve on the fine mesh and the power-spectrum binning.
//
// Mesh layout: real rho / Phi as rows of N floats with row stride S = N + 4
// (z-major, then y); in place, the r2c result is rows of N/2 + 1 complex
// (kx = 0..N/2) with complex stride S/2.  Transforms are unnormalised; the
// 1/N^3 of the inverse is folded into the Green's function.
//
// Each kernel transforms one tile of NC = 16 columns of length n in shared
// memory with a mixed-radix (8, 4, 2, 3) Stockham autosort FFT: every pass
// reads each element once and writes it once, through registers.
//   x sweep : 16 rows per CTA, r2c / c2r by the even-odd packing into an
//             N/2-point complex transform (layout [k][row], XOR-swizzled so
//             row-wise and column-wise accesses are both conflict-free)
//   y sweep : 16 consecutive kx columns of one z-slab
//   z sweep : 16 consecutive kx columns of one ky line; forward, times
//             -(3/2) Om / k^2 / W(k)^p / N^3, inverse, in one pass.
#include <cmath>

#include "kernels.h"

namespace cube {

namespace {

constexpr int NC = 16;          // columns per tile
constexpr int LOG_NC = 4;
constexpr int FFT_T = 512;      // threads per CTA of the column (y, z) sweeps
constexpr int XFFT_T = 256;     // threads per CTA of the row (x) sweeps

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Tile layout: element k of column (row) c at k NC + c, or, swizzled (x
// sweeps), at k NC + (c ^ ((k ^ (k >> 3)) mod NC)).  The swizzle keeps both
// thread mappings bank-conflict free: one k across the 16 columns, and one
// column across 16 values of k, whether consecutive or with the strides of
// the Stockham passes (checked exhaustively for n/2 = 128 ... 512).
template <bool SWZ>
__device__ __forceinline__ int sidx(int k, int c) {
    return SWZ ? (k << LOG_NC) + (c ^ ((k ^ (k >> 3)) & (NC - 1))) : (k << LOG_NC) + c;
}

// sidx(k_lo + k_hi, c) from base = sidx(k_lo, c) when the set bits of the
// compile-time k_hi lie above those of k_lo: the swizzle is XOR-linear in k,
// so the sum is base XOR a constant plus a constant (one logic op and an
// immediate offset per access)
template <bool SWZ>
__device__ __forceinline__ int sidx_add(int base, int k_hi) {
    return SWZ ? (base ^ ((k_hi ^ (k_hi >> 3)) & (NC - 1))) + (k_hi << LOG_NC) : base + (k_hi << LOG_NC);
}

constexpr bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

template <int RAD, bool INV>
__device__ __forceinline__ void dft(float2* v) {
    if (RAD == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (RAD == 3) {
        const float h = 0.86602540378443865f;   // sqrt(3)/2
        float2 t1 = cadd(v[1], v[2]);
        float2 t2 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
        float2 d = csub(v[1], v[2]);
        float2 t3 = make_float2(h * d.x, h * d.y);
        float2 r = rot90<INV>(t3);               // -+ i * t3
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, r);
        v[2] = csub(t2, r);
    } else if (RAD == 4) {
        float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        float2 b0 = cadd(v[1], v[3]), b1 = rot90<INV>(csub(v[1], v[3]));
        v[0] = cadd(a0, b0);
        v[1] = cadd(a1, b1);
        v[2] = csub(a0, b0);
        v[3] = csub(a1, b1);
    } else {   // 8 = 2 x 4
        const float r = 0.70710678118654752f;
        float2 a[4], b[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            a[m] = cadd(v[m], v[m + 4]);
            b[m] = csub(v[m], v[m + 4]);
        }
        // b[m] *= w8^m,  w8 = e^{-+ 2 pi i / 8}
        b[1] = INV ? make_float2(r * (b[1].x - b[1].y), r * (b[1].x + b[1].y))
                   : make_float2(r * (b[1].x + b[1].y), r * (b[1].y - b[1].x));
        b[2] = rot90<INV>(b[2]);
        b[3] = INV ? make_float2(-r * (b[3].x + b[3].y), r * (b[3].x - b[3].y))
                   : make_float2(r * (b[3].y - b[3].x), -r * (b[3].x + b[3].y));
        dft<4, INV>(a);
        dft<4, INV>(b);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = a[k];
            v[2 * k + 1] = b[k];
        }
    }
}

// one Stockham pass of radix R over the NC-column tile of length n, span Ns;
// twiddles come from a table of TWN = n * TWM entries e^{-2 pi i k / TWN}
template <int n, int Ns, int R, int TWM, bool INV, bool SWZ, int T = FFT_T>
__device__ __forceinline__ void fft_pass(float2* buf, const float2* tw) {
    constexpr int nq = n / R;
    constexpr int nbf = nq * NC;
    constexpr int KMAX = (nbf + T - 1) / T;
    constexpr int step = TWM * (n / (Ns * R));
    constexpr bool lin = pow2(nq) && pow2(Ns) && pow2(R);   // bit-disjoint element offsets
    float2 v[KMAX][R];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * T;
        if (nbf % T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
            const int base = sidx<SWZ>(j, c);
#pragma unroll
            for (int m = 0; m < R; ++m)
                v[q][m] = buf[lin ? sidx_add<SWZ>(base, m * nq) : sidx<SWZ>(j + m * nq, c)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * T;
        if (nbf % T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
            const int k = j % Ns;
            if (Ns > 1) {                                  // span 1: all twiddles are 1
#pragma unroll
                for (int m = 1; m < R; ++m) {
                    float2 w = tw[k * m * step];
                    if (INV) w.y = -w.y;
                    v[q][m] = cmul(v[q][m], w);
                }
            }
            dft<R, INV>(v[q]);
            const int idxD = (j / Ns) * Ns * R + k;
            const int base = sidx<SWZ>(idxD, c);
#pragma unroll
            for (int m = 0; m < R; ++m)
                buf[lin ? sidx_add<SWZ>(base, m * Ns) : sidx<SWZ>(idxD + m * Ns, c)] = v[q][m];
        }
    }
    __syncthreads();
}

// all passes of a length-n transform, radices 8, 4, 2, 3 taken greedily
template <int n, int Ns, int TWM, bool INV, bool SWZ, int T = FFT_T>
__device__ __forceinline__ void tile_fft(float2* buf, const float2* tw) {
    if constexpr (Ns < n) {
        constexpr int rem = n / Ns;
        constexpr int R = rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : 3;
        static_assert(rem % R == 0, "length must be 2^a 3^b");
        fft_pass<n, Ns, R, TWM, INV, SWZ, T>(buf, tw);
        tile_fft<n, Ns * R, TWM, INV, SWZ, T>(buf, tw);
    }
}

// First pass (span 1, no twiddles) of a column tile straight from global
// memory: column c of element j + m n/R is src[(j + m n/R) rs + (c0 + c) cs],
// zero at or past column ncol.  pack_off > 0: column 0 of the tile (c0 = 0)
// becomes X + i Y, X its own values and Y those of the column pack_off
// further (two real sequences in one complex transform).  The caller's
// cp.async copies (twiddles, tables) are waited for before the closing
// barrier.
// UNR = 1 keeps one butterfly's loads in flight per thread (fewer
// registers); UNR = KMAX issues all of them first (more loads in flight)
template <int n, int R, bool INV, int UNR = 1>
__device__ __forceinline__ void fft_pass_load(float2* buf, const float2* __restrict__ src, int64_t rs, int c0,
                                              int ncol, int64_t cs = 1, int pack_off = 0) {
    constexpr int nq = n / R;
    constexpr int nbf = nq * NC;
    constexpr int KMAX = (nbf + FFT_T - 1) / FFT_T;
#pragma unroll UNR
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * FFT_T;
        if (nbf % FFT_T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
            const bool ok = c0 + c < ncol;
            const float2* p = src + (int64_t)j * rs + (int64_t)(c0 + c) * cs;
            float2 v[R];
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = ok ? p[(int64_t)m * nq * rs] : make_float2(0.f, 0.f);
            if (pack_off > 0 && c0 + c == 0)
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const float2 y = p[(int64_t)m * nq * rs + pack_off];
                    v[m] = make_float2(v[m].x - y.y, v[m].y + y.x);
                }
            dft<R, INV>(v);
#pragma unroll
            for (int m = 0; m < R; ++m) buf[sidx<false>(j * R + m, c)] = v[m];
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

// Last pass of a column tile: results (natural order, element j + m Ns) go
// straight to dst[(j + m Ns) rs + (c0 + c) cs] for columns below ncol, each
// first passed through post(element, column, value).  split_off > 0: column
// 0 of the tile (c0 = 0) holds x + i y of two real sequences; x goes to
// column 0 and y to the column split_off further, both as (value, 0).
// Shared memory is only read: the caller synchronises before reusing it.
template <int n, int Ns, int R, int TWM, bool INV, class Post, int UNR = 1>
__device__ __forceinline__ void fft_pass_store(const float2* buf, const float2* tw, float2* dst, int64_t rs, int c0,
                                               int ncol, Post post, int64_t cs = 1, int split_off = 0) {
    constexpr int nq = n / R;
    static_assert(nq == Ns, "the last pass has span n / R");
    constexpr int nbf = nq * NC;
    constexpr int KMAX = (nbf + FFT_T - 1) / FFT_T;
    constexpr int step = TWM * (n / (Ns * R));
#pragma unroll UNR
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * FFT_T;
        if (nbf % FFT_T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
            float2 v[R];
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = buf[sidx<false>(j + m * nq, c)];
            if (Ns > 1) {
#pragma unroll
                for (int m = 1; m < R; ++m) {
                    float2 w = tw[j * m * step];
                    if (INV) w.y = -w.y;
                    v[m] = cmul(v[m], w);
                }
            }
            dft<R, INV>(v);
            if (split_off > 0 && c0 + c == 0) {
                float2* p = dst + (int64_t)j * rs;
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    p[(int64_t)m * Ns * rs] = make_float2(v[m].x, 0.f);
                    p[(int64_t)m * Ns * rs + split_off] = make_float2(v[m].y, 0.f);
                }
            } else if (c0 + c < ncol) {
                float2* p = dst + (int64_t)j * rs + (int64_t)(c0 + c) * cs;
#pragma unroll
                for (int m = 0; m < R; ++m) p[(int64_t)m * Ns * rs] = post(j + m * Ns, c, v[m]);
            }
        }
    }
}

struct NoPost {
    __device__ __forceinline__ float2 operator()(int, int, float2 v) const { return v; }
};

// passes from span Ns on, the last one through fft_pass_store
template <int n, int Ns, int TWM, bool INV, class Post, int UNR = 1>
__device__ __forceinline__ void tile_fft_to_global(float2* buf, const float2* tw, float2* dst, int64_t rs, int c0,
                                                   int ncol, Post post, int64_t cs = 1, int split_off = 0) {
    constexpr int rem = n / Ns;
    constexpr int R = rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : 3;
    static_assert(rem % R == 0, "length must be 2^a 3^b");
    if constexpr (Ns * R == n) {
        fft_pass_store<n, Ns, R, TWM, INV, Post, UNR>(buf, tw, dst, rs, c0, ncol, post, cs, split_off);
    } else {
        fft_pass<n, Ns, R, TWM, INV, false>(buf, tw);
        tile_fft_to_global<n, Ns * R, TWM, INV, Post, UNR>(buf, tw, dst, rs, c0, ncol, post, cs, split_off);
    }
}

// passes from span Ns up to (not including) the last, in shared memory
template <int n, int Ns, int TWM, bool INV, bool SWZ = false, int T = FFT_T>
__device__ __forceinline__ void tile_fft_but_last(float2* buf, const float2* tw) {
    constexpr int rem = n / Ns;
    constexpr int R = rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : 3;
    if constexpr (Ns * R < n) {
        fft_pass<n, Ns, R, TWM, INV, SWZ, T>(buf, tw);
        tile_fft_but_last<n, Ns * R, TWM, INV, SWZ, T>(buf, tw);
    }
}

template <int n>
constexpr int first_radix() {
    return n % 8 == 0 ? 8 : n % 4 == 0 ? 4 : n % 2 == 0 ? 2 : 3;
}

// first radix of the row transforms: never the whole length, so that the
// first (load) and last (store) passes are distinct
template <int n>
constexpr int x_first_radix() {
    return first_radix<n>() < n ? first_radix<n>() : (n % 4 == 0 && n > 4 ? 4 : 2);
}

template <int n, int ns0 = 1>
constexpr int last_span() {   // span of the last pass of tile_fft<n, ns0, ...>
    int ns = ns0;
    while (true) {
        const int rem = n / ns;
        const int r = rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : 3;
        if (ns * r == n) return ns;
        ns *= r;
    }
}

// last pass in shared memory, each result passed through post(element, column, value)
template <int n, int Ns, int R, int TWM, bool INV, class Post>
__device__ __forceinline__ void fft_pass_post(float2* buf, const float2* tw, Post post) {
    constexpr int nq = n / R;
    constexpr int nbf = nq * NC;
    constexpr int KMAX = (nbf + FFT_T - 1) / FFT_T;
    constexpr int step = TWM * (n / (Ns * R));
    float2 v[KMAX][R];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * FFT_T;
        if (nbf % FFT_T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
#pragma unroll
            for (int m = 0; m < R; ++m) v[q][m] = buf[sidx<false>(j + m * nq, c)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * FFT_T;
        if (nbf % FFT_T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
            if (Ns > 1) {
#pragma unroll
                for (int m = 1; m < R; ++m) {
                    float2 w = tw[j * m * step];
                    if (INV) w.y = -w.y;
                    v[q][m] = cmul(v[q][m], w);
                }
            }
            dft<R, INV>(v[q]);
#pragma unroll
            for (int m = 0; m < R; ++m) buf[sidx<false>(j + m * Ns, c)] = post(j + m * Ns, c, v[q][m]);
        }
    }
    __syncthreads();
}

// The last forward pass (span n / R) and the first inverse pass (span 1)
// of the same radix R touch the same R elements per thread (j + m n/R), so
// they run back to back in registers: forward pass, post(element, column,
// value) (the Green's function), inverse radix-R DFT, written where the
// inverse first pass writes (j R + m).
template <int n, int Ns, int R, int TWM, class Post>
__device__ __forceinline__ void fft_pass_fwd_post_inv(float2* buf, const float2* tw, Post post) {
    constexpr int nq = n / R;
    static_assert(nq == Ns, "the last forward pass has span n / R");
    constexpr int nbf = nq * NC;
    constexpr int KMAX = (nbf + FFT_T - 1) / FFT_T;
    constexpr int step = TWM * (n / (Ns * R));
    float2 v[KMAX][R];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * FFT_T;
        if (nbf % FFT_T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
#pragma unroll
            for (int m = 0; m < R; ++m) v[q][m] = buf[sidx<false>(j + m * nq, c)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * FFT_T;
        if (nbf % FFT_T == 0 || b < nbf) {
            const int c = b & (NC - 1), j = b >> LOG_NC;
#pragma unroll
            for (int m = 1; m < R; ++m) v[q][m] = cmul(v[q][m], tw[j * m * step]);
            dft<R, false>(v[q]);
#pragma unroll
            for (int m = 0; m < R; ++m) v[q][m] = post(j + m * Ns, c, v[q][m]);
            dft<R, true>(v[q]);
#pragma unroll
            for (int m = 0; m < R; ++m) buf[sidx<false>(j * R + m, c)] = v[q][m];
        }
    }
    __syncthreads();
}

// twiddle table into shared memory (asynchronous; waited for with the tile)
__device__ __forceinline__ void load_tw(float2* stw, const float2* tw, int N) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) cp_async8(&stw[i], &tw[i]);
}

// NC-column tile of rows 0..n-1 (row stride `rs` complex) into buf[row][NC]:
// 16-byte copies of column pairs; pairs starting at or past `ncol` are zeroed
// instead of read (the second column of the last pair may be the row's
// padding slot, which exists in memory and is never written back)
__device__ __forceinline__ void load_columns(float2* buf, const float2* src, int n, int64_t rs, int c0, int ncol) {
    for (int q = threadIdx.x; q < n * (NC / 2); q += blockDim.x) {
        const int r = q / (NC / 2), cp = 2 * (q % (NC / 2));
        float2* d = &buf[(r << LOG_NC) + cp];
        if (c0 + cp < ncol) cp_async16(d, src + r * rs + c0 + cp);
        else d[0] = d[1] = make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------ x sweeps
// NC = 16 rows per CTA.  The first and last passes run with threads along
// the row (j fastest), so they read and write global memory in coalesced
// runs; the middle passes run across the 16 rows.

// First pass (span 1) of the n = N/2-point transforms of rows row0 .. row0 +
// NC - 1, straight from global memory.  PACK (c2r): the input row holds the
// half spectrum X[0 .. n] and the transform input is Z[k] = E + i O with
// E = X[k] + X*[n-k], O = W^-k (X[k] - X*[n-k]), W = e^{-2 pi i / N} (twiddles
// read from global memory: the shared copy may still be in flight).
template <int n, int R, bool INV, bool PACK>
__device__ __forceinline__ void xpass_load(float2* buf, const float* mesh, int64_t row0, int S,
                                           const float2* __restrict__ gtw) {
    constexpr int nq = n / R;
    constexpr int nbf = nq * NC;
    constexpr int KMAX = (nbf + XFFT_T - 1) / XFFT_T;
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * XFFT_T;
        if (nbf % XFFT_T == 0 || b < nbf) {
            const int j = b % nq, c = b / nq;
            const float2* row = reinterpret_cast<const float2*>(mesh + (row0 + c) * S);
            float2 v[R];
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const int k = j + m * nq;
                if (!PACK) {
                    v[m] = row[k];
                } else {
                    const float2 xk = row[k], xm = row[n - k];
                    const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);
                    const float2 d = make_float2(xk.x - xm.x, xk.y + xm.y);
                    const float2 o = cmul(cconj(gtw[k]), d);
                    v[m] = make_float2(e.x - o.y, e.y + o.x);
                }
            }
            dft<R, INV>(v);
            const int base = sidx<true>(j * R, c);
#pragma unroll
            for (int m = 0; m < R; ++m) buf[pow2(R) ? sidx_add<true>(base, m) : sidx<true>(j * R + m, c)] = v[m];
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

// Last pass (span n / R) of the row transforms of N = 2n reals, straight to
// the ghosted copy of Phi: every row lands at its place and, within the
// ghost layers, at its periodic images (rows y < 3 also at y + N, y >= N - 2
// also at y - N, the same in z; x < 4 also at x + N, x >= N - 4 at x - N).
template <int n, int Ns, int R, int TWM, bool INV>
__device__ __forceinline__ void xpass_store(const float2* buf, const float2* tw, float* phig, int64_t row0) {
    constexpr int N = 2 * n;
    constexpr int nq = n / R;
    static_assert(nq == Ns, "the last pass has span n / R");
    constexpr int nbf = nq * NC;
    constexpr int KMAX = (nbf + XFFT_T - 1) / XFFT_T;
    constexpr int step = TWM * (n / (Ns * R));
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int b = threadIdx.x + q * XFFT_T;
        if (nbf % XFFT_T == 0 || b < nbf) {
            const int j = b % nq, c = b / nq;
            float2 v[R];
            const int base = sidx<true>(j, c);
#pragma unroll
            for (int m = 0; m < R; ++m)
                v[m] = buf[pow2(nq) ? sidx_add<true>(base, m * nq) : sidx<true>(j + m * nq, c)];
            if (Ns > 1) {
#pragma unroll
                for (int m = 1; m < R; ++m) {
                    float2 w = tw[j * m * step];
                    if (INV) w.y = -w.y;
                    v[m] = cmul(v[m], w);
                }
            }
            dft<R, INV>(v);
            const int64_t r = row0 + c;
            const int z = (int)(r / N), y = (int)(r - (int64_t)z * N);
            // element k = j + m Ns holds reals 2k, 2k + 1; k < 2 only for m = 0,
            // k >= n - 2 only for m = R - 1 (Ns >= 2)
            auto put = [&](int yy, int zz) {
                float2* row = reinterpret_cast<float2*>(phig + phig_index(N, 0, yy, zz));
#pragma unroll
                for (int m = 0; m < R; ++m) row[j + m * Ns] = v[m];
                if (j < 2) row[j + n] = v[0];
                if (j >= Ns - 2) row[j + (R - 1) * Ns - n] = v[R - 1];
            };
            put(y, z);
            const bool gy = y < 3 || y >= N - 2, gz = z < 3 || z >= N - 2;
            if (gy || gz) {                      // rows with periodic images in the ghost layers
                const int y2 = y < 3 ? y + N : y - N, z2 = z < 3 ? z + N : z - N;
                if (gy) put(y2, z);
                if (gz) put(y, z2);
                if (gy && gz) put(y2, z2);
            }
        }
    }
}

// r2c: the N reals of a row as N/2 complex z[k] = x[2k] + i x[2k+1], an
// N/2-point FFT Z, then X[k] = (Z[k] + Z*[h-k])/2 - i W^k (Z[k] - Z*[h-k])/2
template <int N, bool BAT>
__global__ void __launch_bounds__(XFFT_T) k_fft_x_r2c(float* mesh, int S, const float2* __restrict__ tw, Batch bt) {
    extern __shared__ float2 fsm[];
    if constexpr (BAT) {                                     // slot blockIdx.y of a batch
        if (bt.ms && !bt.ms[blockIdx.y].active) return;
        mesh = moved(mesh, slot_member(bt, blockIdx.y) * bt.stride);
    }
    constexpr int h = N / 2;
    float2* stw = fsm;               // [N]
    float2* buf = fsm + N;           // [h][NC]
    load_tw(stw, tw, N);
    const int64_t row0 = (int64_t)blockIdx.x * NC;
    constexpr int R1 = x_first_radix<h>();
    xpass_load<h, R1, false, false>(buf, mesh, row0, S, tw);
    tile_fft<h, R1, 2, false, true, XFFT_T>(buf, stw);
    // X[k] and X[h - k] from Z[k] and Z[h - k], k = 0 .. h / 2: the warps
    // take k < h / 2 of one row at a time, so that (h / 2 a multiple of 16)
    // each half-warp's Z[k] are one 16-element block of the swizzled tile,
    // free of bank conflicts; the self-paired k = h / 2 of the 16 rows last
    for (int t = threadIdx.x; t < (h / 2) * NC + NC; t += XFFT_T) {
        const bool mid = t >= (h / 2) * NC;
        const int k = mid ? h / 2 : t % (h / 2), c = mid ? t - (h / 2) * NC : t / (h / 2);
        float2* dst = reinterpret_cast<float2*>(mesh + (row0 + c) * S);
        const float2 zk = buf[sidx<true>(k % h, c)];
        const float2 zm = buf[sidx<true>((h - k) % h, c)];
        {
            float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            float2 o = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));   // (Z - Z*) / 2
            float2 wo = cmul(stw[k], o);
            dst[k] = make_float2(e.x + wo.y, e.y - wo.x);                         // e - i wo
        }
        if (k != h - k) {
            const int km = h - k;
            float2 e = make_float2(0.5f * (zm.x + zk.x), 0.5f * (zm.y - zk.y));
            float2 o = make_float2(0.5f * (zm.x - zk.x), 0.5f * (zm.y + zk.y));
            float2 wo = cmul(stw[km], o);
            dst[km] = make_float2(e.x + wo.y, e.y - wo.x);
        }
    }
}

// c2r: the packing above inverted inside the first pass, the N/2-point
// inverse FFT, and the last pass writing the row's N reals
template <int N, bool BAT>
__global__ void __launch_bounds__(XFFT_T) k_fft_x_c2r(const float* mesh, int S, const float2* __restrict__ tw,
                                                     float* __restrict__ phig, Batch bt) {
    extern __shared__ float2 fsm[];
    if constexpr (BAT) {                                     // slot blockIdx.y of a batch
        if (bt.ms && !bt.ms[blockIdx.y].active) return;
        const int m = slot_member(bt, blockIdx.y);
        mesh = moved(mesh, m * bt.stride);
        phig = moved(phig, m * bt.stride);
    }
    constexpr int h = N / 2;
    float2* stw = fsm;               // [N]
    float2* buf = fsm + N;           // [h][NC]
    load_tw(stw, tw, N);
    const int64_t row0 = (int64_t)blockIdx.x * NC;
    constexpr int R1 = x_first_radix<h>();
    xpass_load<h, R1, true, true>(buf, mesh, row0, S, tw);
    tile_fft_but_last<h, R1, 2, true, true, XFFT_T>(buf, stw);
    constexpr int Ns = last_span<h, R1>();
    xpass_store<h, Ns, h / Ns, 2, true>(buf, stw, phig, row0);
}

// ------------------------------------------------------------ y sweep
// The tile's first pass reads global memory and its last pass writes it:
// shared memory holds only the intermediate passes.  Columns kx = 0 and
// kx = N/2 are real before the forward sweep and after the inverse one, so
// they share one complex column (x + i y) in tile 0, and N/2 / NC tiles
// cover the N/2 + 1 columns.  Forward, tile 0 separates the two transforms
// by Hermitian symmetry, A(k) = (Z(k) + Z*(N-k)) / 2, B(k) = (Z(k) - Z*(N-k)) / 2i.
template <int N>
constexpr int ntile_x() { return (N / 2 + NC - 1) / NC; }

template <int N, bool INV, bool BAT>
__global__ void __launch_bounds__(FFT_T, N <= 512 ? 2 : 1) k_fft_y(float* mesh, int S, const float2* __restrict__ tw,
                                                                    Batch bt) {
    extern __shared__ float2 fsm[];
    if constexpr (BAT) {                                     // slot blockIdx.z of a batch
        if (bt.ms && !bt.ms[blockIdx.z].active) return;
        mesh = moved(mesh, slot_member(bt, blockIdx.z) * bt.stride);
    }
    constexpr int h = N / 2;
    float2* stw = fsm;
    float2* buf = fsm + N;
    load_tw(stw, tw, N);
    const int Sc = S / 2;
    const int c0 = blockIdx.x * NC;
    float2* slab = reinterpret_cast<float2*>(mesh) + (int64_t)blockIdx.y * N * Sc;
    constexpr int R1 = first_radix<N>(), KMAX1 = (N / R1 * NC + FFT_T - 1) / FFT_T;
    fft_pass_load<N, R1, INV, INV ? 1 : KMAX1>(buf, slab, Sc, c0, h, 1, h);
    if (INV) {
        tile_fft_to_global<N, first_radix<N>(), 1, INV>(buf, stw, slab, Sc, c0, h, NoPost{}, 1, h);
    } else if (blockIdx.x > 0) {
        constexpr int KL = (last_span<N>() * NC + FFT_T - 1) / FFT_T;
        tile_fft_to_global<N, first_radix<N>(), 1, INV, NoPost, KL>(buf, stw, slab, Sc, c0, h, NoPost{});
    } else {
        tile_fft<N, first_radix<N>(), 1, INV, false>(buf, stw);
        for (int t = threadIdx.x; t < N * NC; t += FFT_T) {
            const int c = t & (NC - 1), ky = t >> LOG_NC;
            float2* row = slab + (int64_t)ky * Sc;
            if (c == 0) {
                const float2 zk = buf[sidx<false>(ky, 0)];
                const float2 zm = buf[sidx<false>((N - ky) % N, 0)];
                row[0] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                row[h] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
            } else if (c < h) {
                row[c] = buf[sidx<false>(ky, c)];
            }
        }
    }
}

// ------------------------------------------------------------ z sweep (+ Green)
// Green's function -(3/2) Om / k^2 / W(k)^p / N^3 of one column (kx, ky), kz = z
struct GreenPost {
    const float* sk2;
    const float* swd;
    float g0, ky2, wy;
    int c0, ky, ncol;
    __device__ __forceinline__ float2 operator()(int z, int c, float2 v) const {
        const int kx = c0 + c;
        if (kx >= ncol) return v;
        const float kk = sk2[kx] + ky2 + sk2[z];
        // approximate division: within 2 ulp for kk below 2^126 (here kk < 3 pi^2)
        const float gr = (kx == 0 && ky == 0 && z == 0) ? 0.0f : __fdividef(g0, kk) * (swd[kx] * wy * swd[z]);
        return make_float2(v.x * gr, v.y * gr);
    }
};

// One tile of 16 consecutive kx (0 .. N/2) at one ky.
template <int N, int MODE, bool BAT>   // MODE 0: forward only, 1: forward, Green, inverse
__global__ void __launch_bounds__(FFT_T, N <= 512 ? 2 : 1) k_fft_z(float* mesh, int S, const float2* __restrict__ tw,
                                                 const float* __restrict__ k2, const float* __restrict__ wdec, float g0,
                                                 Batch bt) {
    extern __shared__ float2 fsm[];
    if constexpr (BAT) {                                     // slot blockIdx.z of a batch
        if (bt.ms && !bt.ms[blockIdx.z].active) return;
        mesh = moved(mesh, slot_member(bt, blockIdx.z) * bt.stride);
    }
    constexpr int ncol = N / 2 + 1;
    float2* stw = fsm;
    float2* buf = fsm + N;
    float* sk2 = reinterpret_cast<float*>(buf + N * NC + NC);     // [N]
    float* swd = sk2 + N;                                          // [N]
    load_tw(stw, tw, N);
    const int Sc = S / 2;
    const int64_t zs = (int64_t)N * Sc;
    const int c0 = blockIdx.x * NC, ky = blockIdx.y;
    float2* base = reinterpret_cast<float2*>(mesh) + (int64_t)ky * Sc;
    if (MODE == 1)
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            cp_async4(&sk2[i], &k2[i]);
            cp_async4(&swd[i], &wdec[i]);
        }
    fft_pass_load<N, first_radix<N>(), false>(buf, base, zs, c0, ncol);
    if (MODE == 1) {
        tile_fft_but_last<N, first_radix<N>(), 1, false>(buf, stw);
        constexpr int Ns = last_span<N>();
        const GreenPost gp{sk2, swd, g0, sk2[ky], swd[ky], c0, ky, ncol};
        if constexpr (N / Ns == first_radix<N>()) {     // last forward radix = first inverse radix
            fft_pass_fwd_post_inv<N, Ns, N / Ns, 1>(buf, stw, gp);
            tile_fft_to_global<N, first_radix<N>(), 1, true>(buf, stw, base, zs, c0, ncol, NoPost{});
        } else {
            fft_pass_post<N, Ns, N / Ns, 1, false>(buf, stw, gp);
            tile_fft_to_global<N, 1, 1, true>(buf, stw, base, zs, c0, ncol, NoPost{});
        }
    } else {
        tile_fft_to_global<N, first_radix<N>(), 1, false>(buf, stw, base, zs, c0, ncol, NoPost{});
    }
}

// ------------------------------------------------------------ largest force component
// max over mesh nodes and axes of |8 (f(+1) - f(-1)) - (f(+2) - f(-2))| / 12 of
// the ghosted potential (the FD4 gradient the force gather interpolates), as
// the bits of a non-negative float
__global__ void k_grad_max(const float* __restrict__ phig, int N, unsigned* __restrict__ out_bits) {
    const int64_t n3 = (int64_t)N * N * N;
    const int64_t sy = phig_nx(N), sz = sy * phig_ny(N);
    float m = 0.0f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % N), y = (int)((t / N) % N), z = (int)(t / ((int64_t)N * N));
        const float* c = phig + phig_index(N, x, y, z);
        const float gx = 8.0f * (c[1] - c[-1]) - (c[2] - c[-2]);
        const float gy = 8.0f * (c[sy] - c[-sy]) - (c[2 * sy] - c[-2 * sy]);
        const float gz = 8.0f * (c[sz] - c[-sz]) - (c[2 * sz] - c[-2 * sz]);
        m = fmaxf(m, fmaxf(fabsf(gx), fmaxf(fabsf(gy), fabsf(gz))));
    }
    const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(m / 12.0f));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(out_bits, b);
}

// ------------------------------------------------------------ power spectrum
__global__ void k_pk_bin(const float* __restrict__ mesh, int N, int S, int nbins, double pfac, double kfund,
                         const double* __restrict__ wpk, double* __restrict__ part) {
    extern __shared__ double pacc[];          // [3 * nbins]: weight, weight*|k|, weight*P
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) pacc[i] = 0.0;
    __syncthreads();
    const int Sc = S / 2, ncol = N / 2 + 1;
    const int kz = blockIdx.x;
    const int fz = kz <= N / 2 ? kz : kz - N;
    const float2* plane = reinterpret_cast<const float2*>(mesh) + (int64_t)kz * N * Sc;
    for (int t = threadIdx.x; t < N * ncol; t += blockDim.x) {
        int kx = t % ncol, ky = t / ncol;
        int fy = ky <= N / 2 ? ky : ky - N;
        long long n2 = (long long)kx * kx + (long long)fy * fy + (long long)fz * fz;
        if (n2 == 0) continue;
        long long i = (long long)sqrt((double)n2);
        while (i * i > n2) --i;
        while ((i + 1) * (i + 1) <= n2) ++i;
        if (n2 > i * (i + 1)) ++i;
        if (i < 1 || i > nbins) continue;
        float2 v = plane[(int64_t)ky * Sc + kx];
        double p = ((double)v.x * v.x + (double)v.y * v.y) * pfac * wpk[kx] * wpk[ky] * wpk[kz];
        double wt = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
        int b = (int)(i - 1);
        atomicAdd(&pacc[b], wt);
        atomicAdd(&pacc[nbins + b], wt * kfund * sqrt((double)n2));
        atomicAdd(&pacc[2 * nbins + b], wt * p);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) part[(int64_t)blockIdx.x * 3 * nbins + i] = pacc[i];
}

__global__ void k_pk_reduce(const double* __restrict__ part, int nblocks, int nbins, double* k, double* pk, double* nm) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    double w = 0, ks = 0, ps = 0;
    for (int j = 0; j < nblocks; ++j) {
        const double* p = part + (int64_t)j * 3 * nbins;
        w += p[b];
        ks += p[nbins + b];
        ps += p[2 * nbins + b];
    }
    nm[b] = w;
    k[b] = w > 0 ? ks / w : nan("");
    pk[b] = w > 0 ? ps / w : nan("");
}

__global__ void k_unpad_phig(const float* __restrict__ phig, int N, float* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)N * N * N;
    if (t >= tot) return;
    const int x = (int)(t % N), y = (int)((t / N) % N), z = (int)(t / ((int64_t)N * N));
    out[t] = phig[phig_index(N, x, y, z)];
}

__global__ void k_unpad(const float* __restrict__ mesh, int N, int S, float* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)N * N * N;
    if (t >= tot) return;
    int64_t row = t / N;
    int x = (int)(t - row * N);
    out[t] = mesh[row * S + x];
}

// twiddles (N) + tile (n x NC) + one spare column + Green tables (2 x N floats)
size_t tile_smem(int N, int n) { return (size_t)(N + n * NC + NC) * sizeof(float2) + (size_t)2 * N * sizeof(float); }

template <int N>
struct Sweeps {
    template <bool BAT>
    static void attrs_for() {
        if constexpr (BAT && !(N <= 256)) return;
        else {
        const int big = (int)tile_smem(N, N), half = (int)tile_smem(N, N / 2);
        cudaFuncSetAttribute(k_fft_x_r2c<N, BAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, half);
        cudaFuncSetAttribute(k_fft_x_c2r<N, BAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, half);
        cudaFuncSetAttribute(k_fft_y<N, false, BAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        cudaFuncSetAttribute(k_fft_y<N, true, BAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        cudaFuncSetAttribute(k_fft_z<N, 0, BAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        cudaFuncSetAttribute(k_fft_z<N, 1, BAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        }
    }
    // instances with a member dimension exist for the small meshes, where a
    // step is launch-bound; a batch of larger meshes is launched member by member
    static constexpr bool kBatchable = N <= 256;
    static void attrs() {
        static bool done = false;
        if (done) return;
        attrs_for<false>();
        if constexpr (kBatchable) attrs_for<true>();
        done = true;
    }
    // a batch (several members or a per-member table) takes the instances with a member dimension
    static bool batched(const Batch& bt) { return bt.members > 1 || bt.ms != nullptr; }
    // slot by slot from the host: the members the launch lists
    template <class Fn>
    static void per_member(const Batch& bt, Fn fn) {
        for (int i = 0; i < bt.members; ++i) fn((size_t)slot_member(bt, i) * bt.stride);
    }
    static void x_r2c(const FftPlan& p, float* mesh, int S, cudaStream_t st, const Batch& bt) {
        attrs();
        if constexpr (kBatchable) {
            if (batched(bt)) {
                k_fft_x_r2c<N, true><<<dim3((N * N) / NC, bt.members), XFFT_T, tile_smem(N, N / 2), st>>>(mesh, S,
                                                                                                         p.tw, bt);
                return;
            }
        }
        per_member(bt, [&](size_t o) {
            k_fft_x_r2c<N, false><<<(N * N) / NC, XFFT_T, tile_smem(N, N / 2), st>>>(moved(mesh, o), S, p.tw, kSingle);
        });
    }
    static void y(const FftPlan& p, float* mesh, int S, bool inv, cudaStream_t st, const Batch& bt) {
        attrs();
        const size_t sm = tile_smem(N, N);
        if constexpr (kBatchable) {
            if (batched(bt)) {
                const dim3 gy(ntile_x<N>(), N, bt.members);
                if (inv) k_fft_y<N, true, true><<<gy, FFT_T, sm, st>>>(mesh, S, p.tw, bt);
                else k_fft_y<N, false, true><<<gy, FFT_T, sm, st>>>(mesh, S, p.tw, bt);
                return;
            }
        }
        const dim3 gy(ntile_x<N>(), N);
        per_member(bt, [&](size_t o) {
            if (inv) k_fft_y<N, true, false><<<gy, FFT_T, sm, st>>>(moved(mesh, o), S, p.tw, kSingle);
            else k_fft_y<N, false, false><<<gy, FFT_T, sm, st>>>(moved(mesh, o), S, p.tw, kSingle);
        });
    }
    static void z(const FftPlan& p, float* mesh, int S, float g0, bool green, cudaStream_t st, const Batch& bt) {
        attrs();
        const size_t sm = tile_smem(N, N);
        if constexpr (kBatchable) {
            if (batched(bt)) {
                const dim3 gz((N / 2 + NC) / NC, N, bt.members);
                if (green) k_fft_z<N, 1, true><<<gz, FFT_T, sm, st>>>(mesh, S, p.tw, p.k2, p.wdec, g0, bt);
                else k_fft_z<N, 0, true><<<gz, FFT_T, sm, st>>>(mesh, S, p.tw, p.k2, p.wdec, g0, bt);
                return;
            }
        }
        const dim3 gz((N / 2 + NC) / NC, N);
        per_member(bt, [&](size_t o) {
            if (green) k_fft_z<N, 1, false><<<gz, FFT_T, sm, st>>>(moved(mesh, o), S, p.tw, p.k2, p.wdec, g0, kSingle);
            else k_fft_z<N, 0, false><<<gz, FFT_T, sm, st>>>(moved(mesh, o), S, p.tw, p.k2, p.wdec, g0, kSingle);
        });
    }
    static void x_c2r(const FftPlan& p, float* mesh, int S, float* phig, cudaStream_t st, const Batch& bt) {
        attrs();
        if constexpr (kBatchable) {
            if (batched(bt)) {
                k_fft_x_c2r<N, true><<<dim3((N * N) / NC, bt.members), XFFT_T, tile_smem(N, N / 2), st>>>(mesh, S,
                                                                                                         p.tw, phig, bt);
                return;
            }
        }
        per_member(bt, [&](size_t o) {
            k_fft_x_c2r<N, false><<<(N * N) / NC, XFFT_T, tile_smem(N, N / 2), st>>>(moved(mesh, o), S, p.tw,
                                                                                     moved(phig, o), kSingle);
        });
    }
};

// mesh sizes with compiled sweeps: 2^a and 3 * 2^a from 16 to 1024
#define CUBE_FFT_SIZES(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

}  // namespace

bool fft_size_supported(int N) {
    switch (N) {
#define CASE(n) case n:
        CUBE_FFT_SIZES(CASE)
#undef CASE
        return true;
        default: return false;
    }
}

#define DISPATCH()                                       \
    switch (p.N) {                                       \
        CUBE_FFT_SIZES(DCASE)                            \
        default: break;                                  \
    }

void fft_x_r2c(const FftPlan& p, float* mesh, int S, cudaStream_t st, const Batch& bt) {
#define DCASE(n) case n: Sweeps<n>::x_r2c(p, mesh, S, st, bt); break;
    DISPATCH()
#undef DCASE
}

void fft_y(const FftPlan& p, float* mesh, int S, bool inverse, cudaStream_t st, const Batch& bt) {
#define DCASE(n) case n: Sweeps<n>::y(p, mesh, S, inverse, st, bt); break;
    DISPATCH()
#undef DCASE
}

void fft_z(const FftPlan& p, float* mesh, int S, float g0, bool green, cudaStream_t st, const Batch& bt) {
#define DCASE(n) case n: Sweeps<n>::z(p, mesh, S, g0, green, st, bt); break;
    DISPATCH()
#undef DCASE
}

void fft_x_c2r(const FftPlan& p, float* mesh, int S, float* phig, cudaStream_t st, const Batch& bt) {
#define DCASE(n) case n: Sweeps<n>::x_c2r(p, mesh, S, phig, st, bt); break;
    DISPATCH()
#undef DCASE
}

int pk_blocks(int N) { return N; }

void launch_pk_bin(const FftPlan& p, const float* mesh, int S, int nbins, double pfac, double kfund, double* part,
                   cudaStream_t st) {
    size_t sm = (size_t)3 * nbins * sizeof(double);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_pk_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_pk_bin<<<p.N, 512, sm, st>>>(mesh, p.N, S, nbins, pfac, kfund, p.wpk, part);
}

void launch_pk_reduce(const double* part, int nblocks, int nbins, double* k, double* pk, double* nm, cudaStream_t st) {
    k_pk_reduce<<<(nbins + 127) / 128, 128, 0, st>>>(part, nblocks, nbins, k, pk, nm);
}

void launch_grad_max(const float* phig, int N, unsigned* out_bits, cudaStream_t st) {
    cudaMemsetAsync(out_bits, 0, sizeof(unsigned), st);
    k_grad_max<<<4 * 152, 256, 0, st>>>(phig, N, out_bits);
}

void launch_unpad_phig(const float* phig, int N, float* out, cudaStream_t st) {
    int64_t tot = (int64_t)N * N * N;
    k_unpad_phig<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(phig, N, out);
}

void launch_unpad(const float* mesh, int N, int S, float* out, cudaStream_t st) {
    int64_t tot = (int64_t)N * N * N;
    k_unpad<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(mesh, N, S, out);
}

}  // namespace cube
