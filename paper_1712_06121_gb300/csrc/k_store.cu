// Kernels on the compressed, cell-ordered particle store:
//   encode (Fig. fig.ic, Section 2.3.2), decode (Eqs. x, v), CIC deposit,
//   pass A (decode, CIC gather of -grad Phi, kick, re-encode, drift, new-cell
//   histograms; Figs. update_vp and update_xp first loop), cells (counts,
//   offsets and v_c of the new store from the scanned histograms), pass B
//   (identical drift, stable scatter by new cell,
//   Eq. chi / Eq. nu encode against the new v_c; Fig. update_xp second loop).
//
// Every per-particle pass runs one CTA per storage brick: the brick's cells
// are contiguous in the store, so the CTA reads a contiguous particle range
// and finds each particle's cell by binary search in the brick's offsets.
#include <algorithm>

#include "kernels.h"

namespace cube {

namespace {

constexpr int T_BRICK = 256;                 // threads of the per-brick kernels
constexpr double PI_D = 3.141592653589793;   // nearest double to pi

__device__ __forceinline__ int upper_cell(const unsigned* off, int ncell, unsigned i) {
    // largest c in [0, ncell) with off[c] <= i  (off[ncell] > i)
    int lo = 0, hi = ncell;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Cells of a warp's 32 consecutive particles base + lane, from c0, the cell
// of particle base (off[c0] <= base < off[c0 + 1]; a brick's cells are
// contiguous and in order).  Lane j holds b_j = off[c0 + 1 + j] - base, which
// does not decrease with j, and the cell of particle base + l is
// c0 + #{j : b_j <= l}: a binary search over the lanes through shuffles.
// More than 32 cell starts within the round (empty cells) are finished by a
// walk.  *c_next is the cell of particle base + 32.  All 32 lanes call it,
// converged; every shuffle and vote below runs on all of them.
__device__ __forceinline__ int warp_cells(const unsigned* off, int ncell, unsigned base, int c0, int* c_next) {
    const unsigned lane = threadIdx.x & 31;
    const int cj = c0 + 1 + (int)lane;
    const unsigned b = cj < ncell ? off[cj] - base : 0xffffffffu;
    int k = 0;
#pragma unroll
    for (int st = 16; st >= 1; st >>= 1)
        k += __shfl_sync(0xffffffffu, b, k + st - 1) <= lane ? st : 0;
    const unsigned b31 = __shfl_sync(0xffffffffu, b, 31);    // by every lane, before any branch
    if (k == 31 && b31 <= lane) k = 32;
    int c = c0 + k;
    if (k == 32)
        while (c + 1 < ncell && off[c + 1] <= base + lane) ++c;
    const unsigned m = __ballot_sync(0xffffffffu, b <= 32u);
    int cn = c0 + __popc(m);
    if (m == 0xffffffffu)
        while (cn + 1 < ncell && off[cn + 1] <= base + 32) ++cn;
    *c_next = cn;
    return c;
}

// brick of a CTA launched on the (nb, nb, nb x members) grid: its
// coordinates and storage rank; *m the member of a batch
template <bool BAT>
__device__ __forceinline__ int grid_brick(const Geo& g, int* bx, int* by, int* bz, int* m) {
    *m = BAT ? (int)blockIdx.z / g.nb : 0;
    *bx = blockIdx.x;
    *by = blockIdx.y;
    *bz = (int)blockIdx.z - *m * g.nb;
    return *bx + g.nb * (*by + g.nb * *bz);
}

// One axis of the flattened (cell, brick) slot of a halo cell (flat_slot),
// for the brick at coordinate `me` on that axis and halo coordinate e in
// [0, Bh): the cell's home brick coordinate (bits 0-7), its coordinate in
// that brick (8-11), this brick's rank among the cell's candidate bricks
// (12-15), the number of candidates (16-19) and of candidate slots before
// the cell (20-23).  Bricks of 1, 2 or 4 cells and at most 256 bricks per
// side keep every field in range.
__device__ __forceinline__ unsigned halo_axis_desc(const Geo& g, int me, int e) {
    const int c = wrap1(me * g.B - 1 + e, g.Nc);
    const int lx = c & (g.B - 1), hbc = c >> g.lB;
    const int lo = lx == 0 ? wrap1(hbc - 1, g.nb) : -1;
    const int hi = lx == g.B - 1 ? wrap1(hbc + 1, g.nb) : -1;
    const int r = (hbc < me) + (lo >= 0 && lo < me) + (hi >= 0 && hi < me);
    return (unsigned)hbc | ((unsigned)lx << 8) | ((unsigned)r << 12) | ((unsigned)ncand(lx, g.B) << 16) |
           ((unsigned)ncand_before(lx) << 20);
}

// the flattened slot (flat_slot) and the storage rank (cell_rank) of the
// halo cell whose three axes have descriptions ax, ay, az
__device__ __forceinline__ void halo_slot(const Geo& g, unsigned ax, unsigned ay, unsigned az, int64_t* slot,
                                          int* rank_L) {
    const int S1 = g.Bh, S2 = S1 * S1;
    const int hb = (int)(ax & 255u) + g.nb * ((int)(ay & 255u) + g.nb * (int)(az & 255u));
    const int nc0 = (ax >> 16) & 15, nc1 = (ay >> 16) & 15, nc2 = (az >> 16) & 15;
    const int pre = (int)((az >> 20) & 15) * S2 + nc2 * ((int)((ay >> 20) & 15) * S1 + nc1 * (int)((ax >> 20) & 15));
    const int rank = ((int)((az >> 12) & 15) * nc1 + (int)((ay >> 12) & 15)) * nc0 + (int)((ax >> 12) & 15);
    *slot = (int64_t)hb * (S2 * S1) + pre + rank;
    *rank_L = (hb << (3 * g.lB)) + (int)((ax >> 8) & 15) + ((int)((ay >> 8) & 15) << g.lB) +
              ((int)((az >> 8) & 15) << (2 * g.lB));
}

__device__ __forceinline__ void brick_coords(const Geo& g, int brick, int* bx, int* by, int* bz) {
    *bx = brick % g.nb;
    *by = (brick / g.nb) % g.nb;
    *bz = brick / (g.nb * g.nb);
}

__device__ double block_sum_double(double v, double* sh) {
    // fixed-shape tree: deterministic for a given block size
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) s += sh[i];
    __syncthreads();
    return s;
}

__device__ __forceinline__ double snap_sigma_dev(double x) {
    // nearest 2^(m/16) in log2 (ties up), floor 2^-30
    x = fmax(x, 9.313225746154785e-10);
    double m = floor(16.0 * log2(x) + 0.5);
    return exp2(m / 16.0);
}

// ------------------------------------------------------------------ encode
template <int NX>
__global__ void k_encode_keys(Geo g, const float* __restrict__ pos, const float* __restrict__ vel,
                              unsigned* __restrict__ key, unsigned* __restrict__ val, unsigned* counts,
                              long long* vsum, unsigned* flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Np) return;
    const int nbits = 8 * NX;
    const long long tot = (long long)g.Nc << nbits;
    const float scale = ldexpf(1.0f, nbits - g.r);
    int cell[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float x = pos[d * g.Np + i];
        if (!isfinite(x)) { bad = true; x = 0.0f; }
        long long bf = __float2ll_rd(x * scale);
        bf %= tot;
        if (bf < 0) bf += tot;
        cell[d] = (int)(bf >> nbits);
    }
    unsigned k = (unsigned)cell_rank(g, cell[0], cell[1], cell[2]);
    key[i] = k;
    val[i] = (unsigned)i;
    atomicAdd(&counts[k], 1u);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float v = vel[d * g.Np + i];
        if (!isfinite(v)) { bad = true; v = 0.0f; }
        atomicAdd(reinterpret_cast<unsigned long long*>(&vsum[(int64_t)d * g.Ncc + k]),
                  (unsigned long long)vel_fix(v));
    }
    if (bad) atomicOr(flags, ERR_NONFINITE);
}

__global__ void k_vc_finalize(int ncc, const unsigned* __restrict__ counts, const long long* __restrict__ vsum,
                              float* __restrict__ vc) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncc) return;
    unsigned n = counts[c];
#pragma unroll
    for (int d = 0; d < 3; ++d) vc[(int64_t)d * ncc + c] = vel_unfix_mean(vsum[(int64_t)d * ncc + c], n);
}

__global__ void k_encode_sigma(Geo g, const float* __restrict__ vel, const unsigned* __restrict__ key,
                               const float* __restrict__ vc, float* __restrict__ part) {
    __shared__ double sh[32];
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.Np; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned k = key[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float v = vel[d * g.Np + i];
            if (!isfinite(v)) v = 0.0f;
            float e = v - vc[(int64_t)d * g.Ncc + k];
            acc = __fmaf_rn(e, e, acc);
        }
    }
    double s = block_sum_double((double)acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = (float)s;
}

__global__ void k_sigma_finalize(const float* __restrict__ part, int nparts, double count, double ratio,
                                 double fixed, double* sigma_out, Batch bt) {
    __shared__ double sh[32];
    const int slot = blockIdx.x;                             // slot of a batch
    if (bt.ms) {
        if (!bt.ms[slot].active) return;
        ratio = bt.ms[slot].ratio;
    }
    const int m = slot_member(bt, slot);
    part = moved(part, m * bt.stride);
    sigma_out = moved(sigma_out, m * bt.stride);
    // strided FP32 sums per thread (coalesced loads, fixed order), then a fixed tree in FP64
    float acc = 0.0f;
#pragma unroll 8
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
    double s = block_sum_double((double)acc, sh);
    if (threadIdx.x == 0) {
        double x = fixed > 0.0 ? fixed : sqrt(s / count) * ratio;
        *sigma_out = snap_sigma_dev(x);
    }
}

// decode table, thresholds, starting-guess constants and (1-byte codes,
// single block) the bucket table for the codec scale sg
__device__ void codec_tables_body(int lim, const double* __restrict__ tanv, const double* __restrict__ tanh_,
                                  double sg, float* __restrict__ dec, float* __restrict__ thr,
                                  float* __restrict__ est, unsigned char* __restrict__ vtab,
                                  unsigned char* __restrict__ vdel) {
    const double s = sqrt(PI_D / (2.0 * sg * sg));
    const double gam = sqrt(2.0 * sg * sg / PI_D);
    const double m = (double)(2 * lim + 1);
    const VelApprox va{(float)(PI_D / (2.0 * m)), (float)gam, 2 * lim + 1};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= lim + 1; k += gridDim.x * blockDim.x) {
        int ddec = 0, dthr = 0;                          // corrections of the 2-byte tables (vdel)
        if (k == 0) {
            dec[lim] = 0.0f;
            thr[0] = 0.0f;
            est[0] = (float)s;
            est[1] = (float)(m / PI_D);
            est[3] = va.c;
            est[4] = va.gam;
        } else if (k <= lim) {
            float dv = (float)(tanv[k] * gam);
            dec[lim + k] = dv;
            dec[lim - k] = -dv;
            const float tv = __double2float_ru(tanh_[k] / s);
            thr[k] = tv;
            if (vdel) {
                ddec = __float_as_int(dv) - __float_as_int(tan_half_steps(2 * k, va));
                dthr = __float_as_int(tv) - __float_as_int(tan_half_steps(2 * k - 1, va));
            }
        } else {
            thr[lim + 1] = __int_as_float(0x7f800000);   // +inf
        }
        if (vdel) vdel[k] = vdelta_pack(ddec, dthr);
    }
    if (vtab) {   // 1-byte codes (lim < 256), one block: the bucket table of nu_from_table
        __shared__ float sthr[256];
        __syncthreads();
        for (int k = threadIdx.x; k <= lim; k += blockDim.x) sthr[k] = thr[k];
        __syncthreads();
        const int key0 = (int)(__float_as_uint(sthr[1]) >> (23 - VT_B)) - 1;   // first bucket lies below thr[1]
        if (threadIdx.x == 0) est[2] = __int_as_float(key0);
        for (int i = threadIdx.x; i < VT_N; i += blockDim.x) {
            const float A = __uint_as_float((unsigned)(key0 + i) << (23 - VT_B));
            int lo = 0, hi = lim;                       // number of thresholds thr[1..lim] <= A
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sthr[mid] <= A) lo = mid;
                else hi = mid - 1;
            }
            vtab[i] = (unsigned char)lo;
        }
    }
}

__global__ void k_codec_tables(int lim, const double* __restrict__ tanv, const double* __restrict__ tanh_,
                               const double* __restrict__ sigma, float* __restrict__ dec, float* __restrict__ thr,
                               float* __restrict__ est, unsigned char* __restrict__ vtab,
                               unsigned char* __restrict__ vdel, Batch bt) {
    const int slot = blockIdx.y;                             // slot of a batch
    if (bt.ms && !bt.ms[slot].active) return;
    const size_t o = slot_member(bt, slot) * bt.stride;
    codec_tables_body(lim, moved(tanv, o), moved(tanh_, o), *moved(sigma, o), moved(dec, o), moved(thr, o),
                      moved(est, o), moved(vtab, o), moved(vdel, o));
}

template <int NX, int NV>
__global__ void k_encode_scatter(Geo g, const float* __restrict__ pos, const float* __restrict__ vel,
                                 const unsigned* __restrict__ id_in, const unsigned* __restrict__ key,
                                 const unsigned* __restrict__ perm, const float* __restrict__ vc,
                                 const float* __restrict__ thr, const float* __restrict__ est, StoreDev s) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.Np) return;
    const int64_t i = perm[j];
    const unsigned k = key[j];
    if (i >= g.Np || k >= (unsigned)g.Ncc) return;      // only if the sort went wrong
    const int nbits = 8 * NX;
    const long long tot = (long long)g.Nc << nbits;
    const float scale = ldexpf(1.0f, nbits - g.r);
    const float e0 = est[0], e1 = est[1];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float x = pos[d * g.Np + i];
        if (!isfinite(x)) x = 0.0f;
        long long bf = __float2ll_rd(x * scale);
        bf %= tot;
        if (bf < 0) bf += tot;
        int chi = (int)(bf & ((1 << nbits) - 1)) - (1 << (nbits - 1));
        store_code<NX>(s.chi, d * g.Np + j, chi);
        float v = vel[d * g.Np + i];
        if (!isfinite(v)) v = 0.0f;
        float dd = v - vc[(int64_t)d * g.Ncc + k];
        int nu = nu_from_thresholds(dd, thr, g.nulim, nu_estimate(dd, e0, e1));
        store_code<NV>(s.nu, d * g.Np + j, nu);
    }
    if (s.id) store_pid(s.id, (unsigned)j, g.nid, id_in ? id_in[i] : (unsigned)i);
}

// ------------------------------------------------------------------ decode
template <int NX, int NV>
__global__ void __launch_bounds__(T_BRICK) k_decode(Geo g, StoreDev s, const float* __restrict__ dec,
                                                    float* __restrict__ pos, float* __restrict__ vel,
                                                    unsigned* __restrict__ id) {
    extern __shared__ unsigned sm_off[];
    const int nbc = g.B * g.B * g.B;
    const int L0 = blockIdx.x * nbc;
    for (int c = threadIdx.x; c <= nbc; c += blockDim.x) sm_off[c] = s.offsets[L0 + c];
    __syncthreads();
    int bx, by, bz;
    brick_coords(g, blockIdx.x, &bx, &by, &bz);
    const int nbits = 8 * NX, half = 1 << (nbits - 1);
    const double pscale = ldexp(1.0, g.r - nbits - 1);
    const unsigned np_ = (unsigned)g.Np;
    const unsigned q1 = min(sm_off[nbc], np_);
    for (unsigned i = min(sm_off[0], q1) + threadIdx.x; i < q1; i += blockDim.x) {
        int lc = upper_cell(sm_off, nbc, i);
        int l[3] = {lc & (g.B - 1), (lc >> g.lB) & (g.B - 1), lc >> (2 * g.lB)};
        int c[3] = {bx * g.B + l[0], by * g.B + l[1], bz * g.B + l[2]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int Q = 2 * (load_code<NX>(s.chi, d * g.Np + i) + half) + 1;
            long long q = ((long long)c[d] << (nbits + 1)) + Q;
            pos[d * g.Np + i] = __double2float_rn((double)q * pscale);
            int nu = load_nu<NV>(s.nu, d * g.Np + i, g.nulim);
            vel[d * g.Np + i] = s.vc[(int64_t)d * g.Ncc + L0 + lc] + dec[nu + g.nulim];
        }
        if (id) id[i] = s.id ? load_pid(s.id, i, g.nid) : i;
    }
}

// largest |p| over particles and axes of the store (momenta as decoded,
// v_c + tan-table offset), as the bits of a non-negative float (order-
// preserving as unsigned)
template <int NV>
__global__ void __launch_bounds__(T_BRICK) k_max_speed(Geo g, StoreDev s, const float* __restrict__ dec,
                                                       unsigned* __restrict__ vmax_bits, Batch bt) {
    extern __shared__ unsigned sm_off[];
    {                                                        // member of slot blockIdx.y of a batch
        const size_t o = slot_member(bt, blockIdx.y) * bt.stride;
        s = moved(s, o);
        dec = moved(dec, o);
        vmax_bits = moved(vmax_bits, o);
    }
    const int nbc = g.B * g.B * g.B;
    const int L0 = blockIdx.x * nbc;
    for (int c = threadIdx.x; c <= nbc; c += blockDim.x) sm_off[c] = s.offsets[L0 + c];
    __syncthreads();
    const unsigned q1 = min(sm_off[nbc], (unsigned)g.Np);
    float m = 0.0f;
    for (unsigned i = min(sm_off[0], q1) + threadIdx.x; i < q1; i += blockDim.x) {
        const int lc = upper_cell(sm_off, nbc, i);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int nu = load_nu<NV>(s.nu, d * g.Np + i, g.nulim);
            m = fmaxf(m, fabsf(s.vc[(int64_t)d * g.Ncc + L0 + lc] + dec[nu + g.nulim]));
        }
    }
    block_max_to(__float_as_uint(m), vmax_bits);
}

// ------------------------------------------------------------------ CIC deposit
// Owner computes: a CTA produces the density of its brick's fine nodes
// [o, o + F)^3 from the particles of the brick's cells and of the one-cell
// layer below it (a particle in fine cell i also feeds node i + 1).  Weights
// are integers (numerators over 2^s per axis) summed in int64, so the result
// is exact and independent of the summation order; rho = m * sum * 2^(-3s).
__device__ __forceinline__ float node_value(unsigned lo, unsigned hi) {
    return hi ? __ull2float_rn(((unsigned long long)hi << 32) | lo) : u32_to_float_rn(lo);
}

// slots of the per-particle cell table: bricks whose particles and layer
// fit look their cell up in it, larger ones (crowded late epochs) search
constexpr int DEP_QCAP = 2048;

// words of the deposit's node sums: the padded 32-bit tile of the common
// case, (F + 8) x (F + 2)^2 words, or F^3 {lo, hi} pairs, whichever is larger
__host__ __device__ __forceinline__ int dep_acc_words(int F) {
    const int fast = (F + 8) * (F + 2) * (F + 2);
    return fast > 2 * F * F * F ? fast : 2 * F * F * F;
}

template <int NX, int FC, bool BAT>
__global__ void __launch_bounds__(T_BRICK) k_deposit(Geo g, StoreDev s, float* __restrict__ mesh, float fscale,
                                                     Batch bt) {
    extern __shared__ unsigned long long dep_smem[];
    // FC > 0: the brick side in fine cells is the compile-time FC, else g.F
    const int lF = FC == 16 ? 4 : FC == 8 ? 3 : FC == 4 ? 2 : g.lF, F = 1 << lF, F3 = 1 << (3 * lF);
    const int E = g.B + 1, E3 = E * E * E;
    // node sums (block-uniform choice): when no sum can exceed 32 bits
    // ("small"), a padded tile of 32-bit words covering x in [-4, F + 4) and
    // y, z in [-1, F], so every corner of every contributing particle lies
    // inside it (no range checks) and rows start on 16-byte boundaries; else
    // [F3] {lo, hi} pairs over the brick's own nodes
    unsigned* acc = reinterpret_cast<unsigned*>(dep_smem);
    unsigned* cstart = acc + dep_acc_words(F);                       // [E3]
    unsigned* cpref = cstart + E3;                                   // [E3 + 1]
    int* cpack = reinterpret_cast<int*>(cpref + E3 + 1);             // [E3] packed cell offsets
    unsigned char* qcell = reinterpret_cast<unsigned char*>(cpack + E3);   // [DEP_QCAP] cell of each slot
    __shared__ unsigned wsum[T_BRICK / 32];
    int bx, by, bz, m;
    grid_brick<BAT>(g, &bx, &by, &bz, &m);
    if constexpr (BAT) {                                     // slot m of a batch
        if (bt.ms && !bt.ms[m].active) return;
        m = slot_member(bt, m);
        s = moved(s, m * bt.stride);
        mesh = moved(mesh, m * bt.stride);
    }
    const int c0[3] = {bx * g.B, by * g.B, bz * g.B};
    // the cells of the brick and of its one-cell layer below (E^3 <= 125 <=
    // one per thread), their particle counts scanned across the block
    unsigned cnt = 0;
    const int t = threadIdx.x;
    if (t < E3) {
        int ec[3];
        split3(t, E, div_magic(E), ec);
        const int lx = ec[0] - 1, ly = ec[1] - 1, lz = ec[2] - 1;
        const int L = cell_rank(g, wrap1(c0[0] + lx, g.Nc), wrap1(c0[1] + ly, g.Nc), wrap1(c0[2] + lz, g.Nc));
        const unsigned a = s.offsets[L];
        cstart[t] = a;
        cnt = s.offsets[L + 1] - a;
        cpack[t] = (lx + 1) | ((ly + 1) << 8) | ((lz + 1) << 16);
    }
    // node sums cleared while the offsets are in flight (both layouts)
    for (int u = threadIdx.x; u < dep_acc_words(F) / 4; u += blockDim.x)
        reinterpret_cast<uint4*>(acc)[u] = make_uint4(0u, 0u, 0u, 0u);
    {
        const int lane = t & 31, wp = t >> 5;
        unsigned v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[wp] = v;
        __syncthreads();
        for (int k = 0; k < wp; ++k) v += wsum[k];
        if (t < E3) {
            cpref[t + 1] = v;
            // this cell's slots of the per-particle cell table (used when
            // the brick's total fits it), before the barrier that publishes
            // the scan
            if (E3 <= 256)
                for (unsigned q = v - cnt, qe = min(v, (unsigned)DEP_QCAP); q < qe; ++q) qcell[q] = (unsigned char)t;
        }
        if (t == 0) cpref[0] = 0;
    }
    __syncthreads();
    const int nbits = 8 * NX, half = 1 << (nbits - 1);
    const int sb = g.sbits, wmask = (1 << sb) - 1, wone = 1 << sb;
    const unsigned total = min(cpref[E3], (unsigned)g.Np);   // bounded even for inconsistent offsets
    // a node's 32-bit sum of 1-byte-code weights (each < 2^(3 s)) cannot wrap
    // when fewer than 2^(32 - 3 s) particles feed the brick
    const bool small = 3 * sb < 32 && total < (1u << (32 - 3 * sb));
    const int ws = small ? 0 : 1;                                   // log2 words per node
    const bool table = total <= (unsigned)DEP_QCAP && E3 <= 256;    // block-uniform
    const int ox = c0[0] * g.R, oy = c0[1] * g.R, oz = c0[2] * g.R;
    if (NX == 1 && small && table) {
        // the common case: padded 32-bit tile, node (x, y, z) of the brick at
        // (x + 4) + DX ((y + 1) + DY (z + 1)); a particle's 8 corners at fixed
        // offsets from its base node, no range checks
        const int DX = F + 8, DY = F + 2, DXY = DX * DY;
        const int8_t* cx = reinterpret_cast<const int8_t*>(s.chi);
        const int8_t* cy = cx + g.Np;
        const int8_t* cz = cy + g.Np;
        const int shift = sb;
        // the next round's cell and codes are requested before this round's atomics
        int tn = 0, xn = 0, yn = 0, zn = 0;
        bool okn = false;
        auto fetch = [&](unsigned qq) {
            tn = qcell[qq];
            const unsigned ii = cstart[tn] + (qq - cpref[tn]);
            okn = ii < (unsigned)g.Np;
            if (okn) {
                xn = cx[ii];
                yn = cy[ii];
                zn = cz[ii];
            }
        };
        if (threadIdx.x < total) fetch(threadIdx.x);
        for (unsigned q = threadIdx.x; q < total; q += blockDim.x) {
            const int tc = tn, chx = xn, chy = yn, chz = zn;
            const bool ok = okn;
            if (q + blockDim.x < total) fetch(q + blockDim.x);
            if (!ok) continue;
            const int pk = cpack[tc];
            // Q = 2 (chi + 128) + 1: fine cell (Q >> sb) inside the coarse cell, weight Q & wmask
            const int Qx = 2 * chx + 257, Qy = 2 * chy + 257, Qz = 2 * chz + 257;
            const int nx = ((pk & 255) - 1) * g.R + (Qx >> shift);
            const int ny = (((pk >> 8) & 255) - 1) * g.R + (Qy >> shift);
            const int nz = ((pk >> 16) - 1) * g.R + (Qz >> shift);
            // a particle of the layer below more than one fine cell from the brick feeds none of its nodes
            if (min(nx, min(ny, nz)) < -1) continue;
            const unsigned wxn = Qx & wmask, wxm = wone - wxn;
            const unsigned wyn = Qy & wmask, wym = wone - wyn;
            const unsigned wzn = Qz & wmask, wzm = wone - wzn;
            const unsigned w00 = wym * wzm, w10 = wyn * wzm, w01 = wym * wzn, w11 = wyn * wzn;
            unsigned* a = acc + (nx + 4) + DX * ((ny + 1) + DY * (nz + 1));
            atomicAdd(a, wxm * w00);
            atomicAdd(a + 1, wxn * w00);
            atomicAdd(a + DX, wxm * w10);
            atomicAdd(a + DX + 1, wxn * w10);
            atomicAdd(a + DXY, wxm * w01);
            atomicAdd(a + DXY + 1, wxn * w01);
            atomicAdd(a + DXY + DX, wxm * w11);
            atomicAdd(a + DXY + DX + 1, wxn * w11);
        }
        __syncthreads();
        // the brick's rows (32-bit offsets: N^2 S < 2^31 for N <= 1024)
        float* mbase = mesh + ((int64_t)oz * g.N + oy) * g.S + ox;
        for (int t4 = threadIdx.x; t4 < F3 / 4; t4 += blockDim.x) {
            const int t = 4 * t4;
            const int x = t & (F - 1), y = (t >> lF) & (F - 1), z = t >> (2 * lF);
            const uint4 v = *reinterpret_cast<const uint4*>(&acc[(x + 4) + DX * ((y + 1) + DY * (z + 1))]);
            float4 f;
            if (max(max(v.x, v.y), max(v.z, v.w)) < (1u << 23)) {     // exact: 2^23 + u is a float
                f = make_float4(__uint_as_float(0x4B000000u | v.x) - 8388608.0f,
                                __uint_as_float(0x4B000000u | v.y) - 8388608.0f,
                                __uint_as_float(0x4B000000u | v.z) - 8388608.0f,
                                __uint_as_float(0x4B000000u | v.w) - 8388608.0f);
            } else {
                f = make_float4(u32_to_float_rn(v.x), u32_to_float_rn(v.y), u32_to_float_rn(v.z),
                                u32_to_float_rn(v.w));
            }
            *reinterpret_cast<float4*>(mbase + (unsigned)((z * g.N + y) * g.S + x)) =
                make_float4(f.x * fscale, f.y * fscale, f.z * fscale, f.w * fscale);
        }
        return;
    }
    for (unsigned q = threadIdx.x; q < total; q += blockDim.x) {
        const int t = table ? (int)qcell[q] : upper_cell(cpref, E3, q);
        const unsigned i = cstart[t] + (q - cpref[t]);
        if (i >= (unsigned)g.Np) continue;
        const int pk = cpack[t];
        const int l[3] = {(pk & 255) - 1, ((pk >> 8) & 255) - 1, (pk >> 16) - 1};
        int nd[3], wn[3], wm[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int Q = 2 * (load_code<NX>(s.chi, d * g.Np + i) + half) + 1;
            nd[d] = l[d] * g.R + (Q >> sb);
            wn[d] = Q & wmask;
            wm[d] = wone - wn[d];
        }
        // a particle of the layer below more than one fine cell from the brick feeds none of its nodes
        if (nd[0] < -1 || nd[1] < -1 || nd[2] < -1) continue;
        // all 8 corners inside the brick's nodes: no per-corner range checks
        const bool inside = nd[0] >= 0 && nd[1] >= 0 && nd[2] >= 0 && nd[0] < F - 1 && nd[1] < F - 1 && nd[2] < F - 1;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
            const int z = nd[2] + dz;
            if (!inside && (z < 0 || z >= F)) continue;
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const int y = nd[1] + dy;
                if (!inside && (y < 0 || y >= F)) continue;
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = nd[0] + dx;
                    if (!inside && (x < 0 || x >= F)) continue;
                    unsigned* a = &acc[((((z << lF) + y) << lF) + x) << ws];
                    if (NX == 1) {   // weight numerators of 1-byte codes: product < 2^27
                        const unsigned w = (unsigned)(dz ? wn[2] : wm[2]) * (unsigned)(dy ? wn[1] : wm[1]) *
                                           (unsigned)(dx ? wn[0] : wm[0]);
                        if (small) {
                            atomicAdd(a, w);          // the 32-bit sum cannot wrap: no carry
                        } else {
                            const unsigned old = atomicAdd(a, w);
                            if (old + w < old) atomicAdd(a + 1, 1u);
                        }
                    } else {
                        const unsigned long long w = (unsigned long long)(dz ? wn[2] : wm[2]) *
                                                     (unsigned long long)(dy ? wn[1] : wm[1]) *
                                                     (unsigned long long)(dx ? wn[0] : wm[0]);
                        smem_add_u64(a, w);
                    }
                }
            }
        }
    }
    __syncthreads();
    // four consecutive x nodes per thread: one or two 16-byte shared loads,
    // one 16-byte store (F and the row stride S are multiples of 4)
    for (int t4 = threadIdx.x; t4 < F3 / 4; t4 += blockDim.x) {
        const int t = 4 * t4;
        const int x = t & (F - 1), y = (t >> lF) & (F - 1), z = t >> (2 * lF);
        // exact integer sum; one rounding when the scale is a power of two (mass 2^k)
        float4 v;
        if (small) {   // block-uniform: 32-bit sums of nodes t .. t + 3
            const uint4 a = reinterpret_cast<const uint4*>(acc)[t4];
            v = make_float4(u32_to_float_rn(a.x) * fscale, u32_to_float_rn(a.y) * fscale,
                            u32_to_float_rn(a.z) * fscale, u32_to_float_rn(a.w) * fscale);
        } else {
            const uint4 a = reinterpret_cast<const uint4*>(acc)[2 * t4];        // {lo, hi} of nodes t, t + 1
            const uint4 b = reinterpret_cast<const uint4*>(acc)[2 * t4 + 1];    // nodes t + 2, t + 3
            v = make_float4(node_value(a.x, a.y) * fscale, node_value(a.z, a.w) * fscale,
                            node_value(b.x, b.y) * fscale, node_value(b.z, b.w) * fscale);
        }
        *reinterpret_cast<float4*>(&mesh[((int64_t)(oz + z) * g.N + (oy + y)) * g.S + ox + x]) = v;
    }
}

// ------------------------------------------------------------------ pass A
// (bricks of more than PB_BIG particles are listed for pass B's whole-CTA path)
constexpr int PB_BIG = 1024;

// threads of a pass A CTA and the CTAs it keeps resident per SM
constexpr int PA_T = 256;
constexpr int PA_MINB = 4;

// One CTA per brick.  Shared memory: Phi tile of (F + 5)^3 fine nodes
// ([o - 2, o + F + 3) per axis, periodic), brick offsets, the histogram of
// destination cells over the brick and its one-cell halo (Bh^3 cells) with
// fixed-point momentum sums, and (1-byte velocities) the codec tables.
template <int NX, int NV, int FC, bool BAT>
__global__ void __launch_bounds__(PA_T, PA_MINB) k_passA(Geo g, StoreDev s, const float* __restrict__ phig,
                                                      const __grid_constant__ CUtensorMap tmap, int use_tma,
                                                      CodecDev cur, float kick, float dc, StepScratch w,
                                                      DriftDebug dbg, Batch bt) {
    extern __shared__ unsigned char pa_smem[];
    __shared__ __align__(8) unsigned long long tile_bar;
    // Phi tile: T x T rows (y, z: [o - 2, o + F + 3)) of TX = F + 8 nodes
    // (x: [o - 4, o + F + 4)), row stride TS = TX floats, read from the
    // ghosted Phi (no wrap): one TMA box, or 16-byte cp.async chunks
    // FC > 0: the brick side in fine cells is the compile-time FC (every
    // tile offset of the gather becomes an immediate), else g.F
    const int F = FC > 0 ? FC : g.F, T = F + 5, TX = F + 8, TS = TX, T3 = T * T * TS;
    const int nbc = g.B * g.B * g.B, Bh = g.Bh, H3 = Bh * Bh * Bh;
    const unsigned mBh = div_magic(Bh);
    const int lim = g.nulim;
    int bx, by, bz, m;
    const int brick = grid_brick<BAT>(g, &bx, &by, &bz, &m);
    if constexpr (BAT) {                                     // slot m of a batch
        if (bt.ms) {
            if (!bt.ms[m].active) return;
            kick = bt.ms[m].kick;
            dc = bt.ms[m].dc;
        }
        m = slot_member(bt, m);
        const size_t o = m * bt.stride;
        s = moved(s, o);
        phig = moved(phig, o);
        cur = moved(cur, o);
        w = moved(w, o);
    }
    const int ox = bx * F - 4, oy = by * F - 2, oz = bz * F - 2;      // tile origin
    long long* vs = reinterpret_cast<long long*>(pa_smem);                 // [3][H3]
    const unsigned sbase = smem_addr(pa_smem);
    float* tile = reinterpret_cast<float*>(pa_smem + (((sbase + 3 * H3 * 8 + 127) & ~127u) - sbase));   // [T3], 128-byte aligned
    if (use_tma) {
        if (threadIdx.x == 0) mbar_init(&tile_bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&tile_bar, (unsigned)T3 * 4u);
            tma_load_4d(tile, &tmap, ox + PHIG_X0, oy + PHIG_Y0, oz + PHIG_Y0, m, &tile_bar);
        }
    }
    unsigned* hist = reinterpret_cast<unsigned*>(tile + T3);                // [H3]
    unsigned* sm_off = hist + H3;                                           // [nbc + 1]
    float* sdec = reinterpret_cast<float*>(sm_off + nbc + 1);               // NV == 1: [2 lim + 1]
    float* sthr = sdec + (NV == 1 ? 2 * lim + 1 : 0);                       // NV == 1: [lim + 2]
    float* svc = sthr + (NV == 1 ? lim + 2 : 0);                            // [3][nbc]: v_c of the brick
    unsigned char* stab = reinterpret_cast<unsigned char*>(svc + 3 * nbc);  // NV == 1: [VT_N] bucket table
    unsigned char* qcell = stab + (NV == 1 ? VT_N : 0);                     // [DEP_QCAP] cell of each particle
    const float* dec = cur.dec;
    const float* thr = cur.thr;
    int key0 = 0;
    if (NV == 1) {
        for (int t = threadIdx.x; t < 2 * lim + 1; t += blockDim.x) sdec[t] = cur.dec[t];
        for (int t = threadIdx.x; t < lim + 2; t += blockDim.x) sthr[t] = cur.thr[t];
        for (int t = threadIdx.x; t < VT_N / 4; t += blockDim.x)
            reinterpret_cast<unsigned*>(stab)[t] = reinterpret_cast<const unsigned*>(cur.vtab)[t];
        dec = sdec;
        thr = sthr;
        key0 = __float_as_int(cur.est[2]);
    }
    const int L0 = brick * nbc;
    for (int t = threadIdx.x; t < 3 * nbc; t += blockDim.x)
        cp_async4(&svc[t], &s.vc[(int64_t)(t >> (3 * g.lB)) * g.Ncc + L0 + (t & (nbc - 1))]);
    for (int c = threadIdx.x; c <= nbc; c += blockDim.x) sm_off[c] = s.offsets[L0 + c];
    for (int t = threadIdx.x; t < H3; t += blockDim.x) {
        hist[t] = 0u;
        vs[t] = 0;
        vs[H3 + t] = 0;
        vs[2 * H3 + t] = 0;
    }
    // per axis d and halo coordinate e in [0, Bh): the coarse cell's home
    // brick coordinate (bits 0-7), its coordinate in that brick (8-11), this
    // brick's rank among the cell's candidate bricks (12-15), the number of
    // candidates (16-19) and of candidate slots before the cell (20-23); the
    // flattened slot of a halo cell combines the three axes (flat_slot)
    __shared__ unsigned axis_desc[3 * 6];
    if (threadIdx.x < 3 * Bh) {
        const int d = threadIdx.x / Bh, ee = threadIdx.x - d * Bh;
        axis_desc[threadIdx.x] = halo_axis_desc(g, d == 0 ? bx : d == 1 ? by : bz, ee);
    }
    if (!use_tma) {
        // rows of TX = F + 8 nodes start on a 16-byte boundary: 4-node chunks;
        // thread t < RPI * CX owns chunk column cx of rows t / CX, + RPI, ...
        const int CX = TX >> 2, nrow = T * T, RPI = PA_T / CX;
        if (threadIdx.x < RPI * CX) {
            const int cx = threadIdx.x % CX;
            int row = threadIdx.x / CX;
            int z = row / T, y = row - z * T;
            const int dz = RPI / T, dy = RPI - dz * T;
            float* dst = tile + 4 * cx;
            for (; row < nrow; row += RPI) {
                cp_async16(dst + row * TS, phig + phig_index(g.N, ox + 4 * cx, oy + y, oz + z));
                y += dy;
                z += dz;
                if (y >= T) {
                    y -= T;
                    ++z;
                }
            }
        }
    }
    // the brick's particle range, and the first round's codes, requested
    // while the tile is in flight
    const unsigned q1 = min(s.offsets[L0 + nbc], (unsigned)g.Np);
    const unsigned q0 = min(s.offsets[L0], q1);
    unsigned i = q0 + threadIdx.x;
    if (threadIdx.x == 0 && q1 - q0 > (unsigned)PB_BIG) w.big[1 + atomicAdd(w.big, 1)] = brick;
    const CodeRows<NX> chi_r(s.chi, g.Np);
    const CodeRows<NV> nu_r(s.nu, g.Np);
    int nchi[3] = {0, 0, 0}, nnu[3] = {0, 0, 0};
    if (i < q1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            nchi[d] = chi_r.get(d, i);
            nnu[d] = nu_r.get_nu(d, i, lim);
        }
    }
    // the cell of every particle of the brick, when they fit the table,
    // written while the tile is in flight (each thread reads its cells' bounds)
    const bool table = q1 - q0 <= (unsigned)DEP_QCAP;                  // block-uniform
    if (table)
        for (int c = threadIdx.x; c < nbc; c += blockDim.x)
            for (unsigned q = max(s.offsets[L0 + c], q0), qe = min(s.offsets[L0 + c + 1], q1); q < qe; ++q)
                qcell[q - q0] = (unsigned char)c;
    cp_async_wait_all();
    const bool tile_ok = !use_tma || mbar_wait_bounded(&tile_bar, 0);
    if (__syncthreads_or(!tile_ok)) {       // the tile copy never completed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(w.flags, ERR_TIMEOUT);
        mbar_wait_bounded(&tile_bar, 0);
        return;
    }
    const float e0 = cur.est[0], e1 = cur.est[1];
    // 2-byte codes: the decode and threshold tables through their L1-resident corrections
    const VelTables vt{cur.dec, cur.thr, cur.vdel, VelApprox{NV == 2 ? cur.est[3] : 0.0f, NV == 2 ? cur.est[4] : 0.0f,
                                                             2 * lim + 1}, lim};
    const int nbits = 8 * NX, half = 1 << (nbits - 1);
    const int sb = g.sbits, wmask = (1 << sb) - 1;
    // the in-cell CIC weight (Q mod 2^sb) 2^-sb exactly from the bits of
    // 2^(23 - sb) + (Q mod 2^sb) 2^-sb
    const int wexp = (127 + 23 - sb) << 23;
    const float wbase = ldexpf(1.0f, 23 - sb);
    const float dcs = ldexpf(dc, nbits);           // drift in bins of the position code
    const float kick12 = kick * (-1.0f / 12.0f);   // the FD4 sums' 1/12 and the sign of -grad Phi
    float sacc = 0.0f;
    int mig = 0;
    bool migbad = false;
    const int TT = T * TS;   // z stride of the tile
    const int lB = g.lB, bm = g.B - 1;
    for (; i < q1; i += blockDim.x) {
        // this round's codes; the next round's are requested now
        const int cchi[3] = {nchi[0], nchi[1], nchi[2]}, cnu[3] = {nnu[0], nnu[1], nnu[2]};
        if (i + blockDim.x < q1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                nchi[d] = chi_r.get(d, i + blockDim.x);
                nnu[d] = nu_r.get_nu(d, i + blockDim.x, lim);
            }
        }
        const int lc = table ? (int)qcell[i - q0] : upper_cell(sm_off, nbc, i);
        const int l[3] = {lc & bm, (lc >> lB) & bm, lc >> (2 * lB)};
        int Q[3], n[3];
        float w1[3], w0[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Q[d] = 2 * (cchi[d] + half) + 1;
            n[d] = (d == 0 ? 4 : 2) + (l[d] << g.r) + (Q[d] >> sb);
            w1[d] = __int_as_float(wexp | (Q[d] & wmask)) - wbase;
            w0[d] = 1.0f - w1[d];
        }
        // CIC gather of the FD4 gradient (56 nodes, read as 28 pairs of
        // x-adjacent nodes {o, o + 1}).  Near a uniform lattice every node
        // index is even, so a warp's loads would use the 16 even banks only; a
        // particle with odd n_y / 2 reads each pair in the other order, which
        // spreads a warp's loads over all 32 banks.  Columns along y and z
        // keep the swapped order and take the matching x weights (ca, cb);
        // rows along x are put back in order.  Two lines at a time in packed
        // FP32 pairs.
        const int base = (n[2] * T + n[1]) * TS + n[0];
        const int sh = (n[1] >> 1) & 1;
        const float* pa = tile + base + sh;
        const float* pb = tile + base + 1 - sh;
        const float ca = sh ? w1[0] : w0[0], cb = sh ? w0[0] : w1[0];   // x weights of the pa, pb values
        float2 gy2 = make_float2(0.0f, 0.0f), gz2 = make_float2(0.0f, 0.0f), gx2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            float2 r[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) r[k] = make_float2(pa[b * TT + (k - 2) * TS], pb[b * TT + (k - 2) * TS]);
            gy2 = pfma(pk2(b ? w1[2] : w0[2]), fd4_cic_pair(r, w0[1], w1[1]), gy2);   // y columns at z + b
#pragma unroll
            for (int k = 0; k < 6; ++k) r[k] = make_float2(pa[b * TS + (k - 2) * TT], pb[b * TS + (k - 2) * TT]);
            gz2 = pfma(pk2(b ? w1[1] : w0[1]), fd4_cic_pair(r, w0[2], w1[2]), gz2);   // z columns at y + b
            // x rows at (y + a, z + b), a = 0, 1 in the two lanes, in natural order
#pragma unroll
            for (int k = 0; k < 6; k += 2) {
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int o = a * TS + b * TT + (k - 2);
                    const float u = pa[o], v = pb[o];
                    (a ? r[k].y : r[k].x) = sh ? v : u;
                    (a ? r[k + 1].y : r[k + 1].x) = sh ? u : v;
                }
            }
            gx2 = pfma(pmul(make_float2(w0[1], w1[1]), pk2(b ? w1[2] : w0[2])), fd4_cic_pair(r, w0[0], w1[0]), gx2);
        }
        // the gathered sums of 12 dPhi/dx_d; F = -sum / 12 is folded into the kick factor
        const float gsum[3] = {gx2.x + gx2.y, __fmaf_rn(ca, gy2.x, cb * gy2.y), __fmaf_rn(ca, gz2.x, cb * gz2.y)};
        // kick (update_vp): the code is decided on v - v_c + F K = offset + F K,
        // re-encoded against the same v_c; then the drift of the in-cell
        // offset Q / 2^(8n+1) by the decoded momentum, rounded once
        int e[3];
        float pv[3], un[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float vcd = svc[(d << (3 * lB)) + lc];
            const float dd = __fmaf_rn(gsum[d], kick12, NV == 1 ? dec[cnu[d] + lim] : vt.dec(cnu[d]));
            const int nu1 = NV == 1 ? nu_from_table(dd, thr, stab, key0, lim)
                                    : nu_from_tables(dd, vt, nu_estimate(dd, e0, e1));
            nu_r.put(d, i, nu1);
            const float off1 = NV == 1 ? dec[nu1 + lim] : vt.dec(nu1);
            const float p2 = vcd + off1;
            sacc = __fmaf_rn(off1, off1, sacc);
            const int sh1 = drift_bin(Q[d], p2, dcs, &un[d]) >> nbits;
            const int shc = max(-1, min(1, sh1));
            migbad |= sh1 != shc;
            mig |= shc & 1;                        // 1 if the particle changes cell along d
            e[d] = l[d] + shc + 1;
            pv[d] = p2;
        }

        const int ei = e[0] + Bh * (e[1] + Bh * e[2]);
        // per-lane shared-memory atomics (measured faster here than warp aggregation)
        atomicAdd(&hist[ei], 1u);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            smem_add_u64(reinterpret_cast<unsigned*>(&vs[d * H3 + ei]), (unsigned long long)vel_fix(pv[d]));
        if (dbg.cell_old) {
            const int cg[3] = {bx * g.B + l[0], by * g.B + l[1], bz * g.B + l[2]};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                dbg.cell_old[d * g.Np + i] = cg[d];
                dbg.u_new[d * g.Np + i] = ldexpf(un[d], -nbits);
                dbg.p[d * g.Np + i] = pv[d];
                dbg.force[d * g.Np + i] = gsum[d] * (-1.0f / 12.0f);
            }
        }
    }
    if (migbad) atomicOr(w.flags, ERR_MIGRATION);
    // the block's sum of squared offsets (a fixed tree: each warp's shuffle
    // tree, then the warps in order) and whether any particle changed cell,
    // finished by thread 0 after the barrier that also opens the write-out
    __shared__ float red[PA_T / 32];
    __shared__ unsigned redmig[PA_T / 32];
    {
        float v = sacc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        const unsigned wm = __reduce_or_sync(0xffffffffu, (unsigned)mig);
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = v;
            redmig[threadIdx.x >> 5] = wm;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.0f;
        unsigned mm = 0u;
#pragma unroll
        for (int k = 0; k < PA_T / 32; ++k) {
            tot += red[k];
            mm |= redmig[k];
        }
        w.part[brick] = tot;
        if (mm) atomicMax(w.maxmig, (int)mm);
    }
    // each halo cell's slot in the flattened (cell, brick) order and its cell
    // rank, from the per-axis descriptions staged before the particle loop
    for (int t = threadIdx.x; t < H3; t += blockDim.x) {
        const unsigned h = hist[t];
        int ec[3];
        split3(t, Bh, mBh, ec);
        int64_t slot;
        int L;
        halo_slot(g, axis_desc[ec[0]], axis_desc[Bh + ec[1]], axis_desc[2 * Bh + ec[2]], &slot, &L);
        w.ghost[slot] = h;                                   // every slot has exactly one writer
        if (h) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
                atomicAdd(reinterpret_cast<unsigned long long*>(&w.vsum_new[(int64_t)d * g.Ncc + L]),
                          (unsigned long long)vs[d * H3 + t]);
        }
    }
}

// ------------------------------------------------------------------ new cells
// After the exclusive scan of the flattened histograms, a cell's first slot
// holds offset*[c] and its slots span counts*[c] particles.  Also
// v_c* = mean momentum of the cell's new particles (fixed point).
template <bool BAT>
__global__ void k_cells(Geo g, StepScratch w, unsigned* __restrict__ off_new, float* __restrict__ vc_new, Batch bt) {
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= g.Ncc) return;
    if constexpr (BAT) {                                     // slot blockIdx.y of a batch
        if (bt.ms && !bt.ms[blockIdx.y].active) return;
        const int m = slot_member(bt, blockIdx.y);
        w = moved(w, m * bt.stride);
        off_new = moved(off_new, m * bt.stride);
        vc_new = moved(vc_new, m * bt.stride);
    }
    const int nbc = g.B * g.B * g.B;
    const int hb = L / nbc, lc = L - hb * nbc;
    const int l[3] = {lc % g.B, (lc / g.B) % g.B, lc / (g.B * g.B)};
    const int64_t base = flat_base(g, hb, l);
    const int n = ncand(l[0], g.B) * ncand(l[1], g.B) * ncand(l[2], g.B);
    const unsigned off = w.ghost[base];
    const unsigned cnt = w.ghost[base + n] - off;
    off_new[L] = off;
    w.counts_new[L] = cnt;
    if (L == g.Ncc - 1) {
        const unsigned total = w.ghost[(int64_t)g.nbricks * (g.Bh * g.Bh * g.Bh)];
        off_new[g.Ncc] = total;
        if (total != (unsigned)g.Np) atomicOr(w.flags, ERR_COUNT);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) vc_new[(int64_t)d * g.Ncc + L] = vel_unfix_mean(w.vsum_new[(int64_t)d * g.Ncc + L], cnt);
}

// ------------------------------------------------------------------ pass B
// One warp per brick (8 bricks per CTA): the brick's particles are taken 32
// at a time in index order; lanes moving to the same cell get consecutive
// slots in lane order from the cell's running start (match + popc), so the
// new order within a cell is the old index order.  No block barriers.
//
// A brick holding more than PB_BIG particles (clustering: late epochs reach
// ~30x the mean) would make its warp the kernel's tail.  Pass A lists those
// bricks; the first CTAs of the grid take them whole, 256 particles per
// round: each warp's per-cell counts go to a shared table, and a lane's slot
// is the cell's running start + the counts of the lower warps + its rank in
// its warp, which is again the old index order.
constexpr int PB_WARPS = 8;

// what pass B needs of one particle: its new cell in the brick's halo
// region (ei), new position code and momentum
struct PbParticle {
    int ei;
    int chi[3];
    float pv[3];
};

// PID: 4 for 4-byte particle IDs (or none), 0 for the narrow widths of Geo::nid
template <int NX, int NV, int PID>
struct PassB {
    Geo g;
    const StoreDev& sn;
    CodeRows<NX> chi_n;
    CodeRows<NV> nu_n;
    const float* dec;
    const float* thr;
    const unsigned char* stab;
    int key0, lim;
    float dcs, e0, e1;     // dcs: the drift factor in bins of the position code (dc 2^(8n))

    // lc: the particle's coarse cell in the brick; its velocity offsets are
    // read from the table (1-byte codes) or given in coff (2-byte codes, read
    // a round ahead)
    __device__ __forceinline__ PbParticle move(int lc, const float* svc, const int* cchi, const int* cnu,
                                               const float* coff) const {
        const int Bh = g.Bh;
        const int nbits = 8 * NX, half = 1 << (nbits - 1), bmask = (1 << nbits) - 1;
        const int l[3] = {lc & (g.B - 1), (lc >> g.lB) & (g.B - 1), lc >> (2 * g.lB)};
        PbParticle r;
        int e[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int Q = 2 * (cchi[d] + half) + 1;
            const float p2 = svc[(d << (3 * g.lB)) + lc] + (NV == 2 ? coff[d] : dec[cnu[d] + lim]);
            float x;
            const int bin = drift_bin(Q, p2, dcs, &x);
            const int sh = max(-1, min(1, bin >> nbits));
            e[d] = l[d] + sh + 1;
            r.chi[d] = (bin & bmask) - half;
            r.pv[d] = p2;
        }
        r.ei = e[0] + Bh * (e[1] + Bh * e[2]);
        return r;
    }

    __device__ __forceinline__ void put(const PbParticle& q, const float* svn, unsigned pos, unsigned cid,
                                        unsigned* flags) const {
        const int H3 = g.Bh * g.Bh * g.Bh;
        if (pos >= (unsigned)g.Np) {
            atomicOr(flags, ERR_COUNT);
            return;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            chi_n.put(d, pos, q.chi[d]);
            const float dd = q.pv[d] - svn[d * H3 + q.ei];
            nu_n.put(d, pos, NV == 1 ? nu_from_table(dd, thr, stab, key0, lim)
                                     : nu_from_thresholds(dd, thr, lim, nu_estimate(dd, e0, e1)));
        }
        if (sn.id) {
            if (PID == 4) reinterpret_cast<unsigned*>(sn.id)[pos] = cid;
            else store_pid(sn.id, pos, g.nid, cid);
        }
    }
};

// brick offsets, v_c of the brick, running starts of the halo cells (this
// brick's slots of the scanned histograms) and v_c* of the halo region,
// staged by `nthr` threads from thread `t0`
__device__ __forceinline__ void passB_stage(const Geo& g, const StoreDev& so, const unsigned* __restrict__ ghost,
                                            const float* __restrict__ vc_new, int brick, int t0, int nthr,
                                            unsigned* sm_off, unsigned* run, float* svc, float* svn) {
    const int nbc = g.B * g.B * g.B, Bh = g.Bh, H3 = Bh * Bh * Bh;
    const unsigned mBh = div_magic(Bh);
    const int L0 = brick * nbc;
    int bx, by, bz;
    brick_coords(g, brick, &bx, &by, &bz);
    const int bc[3] = {bx, by, bz};
    for (int c = t0; c <= nbc; c += nthr) sm_off[c] = so.offsets[L0 + c];
    for (int t = t0; t < 3 * nbc; t += nthr) svc[t] = so.vc[(int64_t)(t >> (3 * g.lB)) * g.Ncc + L0 + (t & (nbc - 1))];
    // the 3 Bh (<= 18) per-axis descriptions of the halo coordinates, one per
    // lane of every warp, read by the others through shuffles
    const int lane = threadIdx.x & 31;
    unsigned dsc = 0u;
    if (lane < 3 * Bh) {
        const int d = lane / Bh;
        dsc = halo_axis_desc(g, bc[d], lane - d * Bh);
    }
    for (int base = t0 - lane; base < H3; base += nthr) {     // warp-uniform bounds
        const int t = base + lane;
        int e[3];
        split3(min(t, H3 - 1), Bh, mBh, e);
        const unsigned ax = __shfl_sync(0xffffffffu, dsc, e[0]);
        const unsigned ay = __shfl_sync(0xffffffffu, dsc, Bh + e[1]);
        const unsigned az = __shfl_sync(0xffffffffu, dsc, 2 * Bh + e[2]);
        if (t < H3) {
            int64_t slot;
            int L;
            halo_slot(g, ax, ay, az, &slot, &L);
            run[t] = ghost[slot];
#pragma unroll
            for (int d = 0; d < 3; ++d) svn[d * H3 + t] = vc_new[(int64_t)d * g.Ncc + L];
        }
    }
}

template <int NX, int NV, bool BAT, int PID>
__global__ void __launch_bounds__(PB_WARPS * 32, 5) k_passB(Geo g, StoreDev so, StoreDev sn, CodecDev cur, CodecDev next,
                                                        float dc, const unsigned* __restrict__ ghost,
                                                        const float* __restrict__ vc_new, unsigned* flags,
                                                        const int* __restrict__ big, int nbig_ctas, Batch bt) {
    extern __shared__ unsigned pb_smem[];
    const int nbc = g.B * g.B * g.B, H3 = g.Bh * g.Bh * g.Bh;
    const int lim = g.nulim;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (BAT) {                                     // slot blockIdx.y of a batch
        const int slot = blockIdx.y;
        if (bt.ms) {
            if (!bt.ms[slot].active) return;
            dc = bt.ms[slot].dc;
        }
        const size_t o = slot_member(bt, slot) * bt.stride;
        so = moved(so, o);
        sn = moved(sn, o);
        cur = moved(cur, o);
        next = moved(next, o);
        ghost = moved(ghost, o);
        vc_new = moved(vc_new, o);
        flags = moved(flags, o);
        big = moved(big, o);
    }
    const bool big_cta = (int)blockIdx.x < nbig_ctas;
    const int nbig = big_cta ? big[0] : 0;
    if (big_cta && (int)blockIdx.x >= nbig) return;          // no crowded brick left for this CTA
    float* sdec = reinterpret_cast<float*>(pb_smem);                       // NV == 1: [2 lim + 1]
    float* sthr = sdec + (NV == 1 ? 2 * lim + 1 : 0);                       // NV == 1: [lim + 2]
    unsigned char* stab = reinterpret_cast<unsigned char*>(sthr + (NV == 1 ? lim + 2 : 0));   // NV == 1: [VT_N]
    unsigned* wbase = reinterpret_cast<unsigned*>(stab + (NV == 1 ? VT_N : 0));
    // (2-byte codes read the full tables here: the compact form of pass A
    // costs pass B more in instructions than its loads cost in latency)
    PassB<NX, NV, PID> pb{g, sn, CodeRows<NX>(sn.chi, g.Np), CodeRows<NV>(sn.nu, g.Np), cur.dec, next.thr, stab, 0, lim,
                     ldexpf(dc, 8 * NX), next.est[0], next.est[1]};
    const CodeRows<NX> chi_o(so.chi, g.Np);
    const CodeRows<NV> nu_o(so.nu, g.Np);
    if (NV == 1) {
        for (int t = threadIdx.x; t < 2 * lim + 1; t += blockDim.x) sdec[t] = cur.dec[t];
        for (int t = threadIdx.x; t < lim + 2; t += blockDim.x) sthr[t] = next.thr[t];
        for (int t = threadIdx.x; t < VT_N / 4; t += blockDim.x)
            reinterpret_cast<unsigned*>(stab)[t] = reinterpret_cast<const unsigned*>(next.vtab)[t];
        pb.dec = sdec;
        pb.thr = sthr;
        pb.key0 = __float_as_int(next.est[2]);
    }
    if (big_cta) {
        // whole CTA per crowded brick: [nbc + 1] offsets, [H3] running starts,
        // [3][nbc] v_c, [3][H3] v_c*, [PB_WARPS][H3] per-warp cell counts
        unsigned* sm_off = wbase;
        unsigned* run = sm_off + nbc + 1;
        float* svc = reinterpret_cast<float*>(run + H3);
        float* svn = svc + 3 * nbc;
        unsigned* wcnt = reinterpret_cast<unsigned*>(svn + 3 * H3);
        for (int t = threadIdx.x; t < PB_WARPS * H3; t += blockDim.x) wcnt[t] = 0u;
        for (int k = blockIdx.x; k < nbig; k += nbig_ctas) {
            const int brick = big[1 + k];
            __syncthreads();                 // the previous brick's tables are no longer read
            passB_stage(g, so, ghost, vc_new, brick, threadIdx.x, blockDim.x, sm_off, run, svc, svn);
            __syncthreads();
            const unsigned p1 = min(sm_off[nbc], (unsigned)g.Np), p0 = min(sm_off[0], p1);
            for (unsigned base = p0; base < p1; base += blockDim.x) {
                const unsigned i = base + threadIdx.x;
                const bool act = i < p1;
                const unsigned am = __ballot_sync(0xffffffffu, act);
                PbParticle q{};
                unsigned cid = 0, peers = 0;
                int leader = 0;
                if (act) {
                    int cchi[3], cnu[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        cchi[d] = chi_o.get(d, i);
                        cnu[d] = nu_o.get_nu(d, i, lim);
                    }
                    if (sn.id) cid = PID == 4 ? reinterpret_cast<const unsigned*>(so.id)[i] : load_pid(so.id, i, g.nid);
                    float coff[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) coff[d] = NV == 2 ? pb.dec[cnu[d] + lim] : 0.0f;
                    q = pb.move(upper_cell(sm_off, nbc, i), svc, cchi, cnu, coff);
                    peers = __match_any_sync(am, q.ei);
                    leader = __ffs(peers) - 1;
                    if (lane == leader) wcnt[warp * H3 + q.ei] = (unsigned)__popc(peers);
                }
                __syncthreads();
                unsigned start = 0, total = 0;
                bool last = true;
                if (act) {
                    if (lane == leader) {
                        start = run[q.ei];
#pragma unroll
                        for (int v = 0; v < PB_WARPS; ++v) {
                            const unsigned c = wcnt[v * H3 + q.ei];
                            if (v < warp) start += c;
                            if (v > warp && c) last = false;
                            total += c;
                        }
                    }
                    start = __shfl_sync(peers, start, leader);
                }
                __syncthreads();                 // every read of run and wcnt is done
                if (act) {
                    if (lane == leader) {
                        if (last) run[q.ei] += total;
                        wcnt[warp * H3 + q.ei] = 0u;
                    }
                    pb.put(q, svn, start + (unsigned)__popc(peers & ((1u << lane) - 1u)), cid, flags);
                }
            }
        }
        return;
    }
    __syncthreads();
    const int brick = ((int)blockIdx.x - nbig_ctas) * PB_WARPS + warp;
    if (brick >= g.nbricks) return;
    const int L0 = brick * nbc;
    const unsigned p1 = min(so.offsets[L0 + nbc], (unsigned)g.Np), p0 = min(so.offsets[L0], p1);
    if (p1 - p0 > (unsigned)PB_BIG) return;              // a crowded brick: taken by a whole CTA
    unsigned* sm_off = wbase + warp * (4 * nbc + 1 + 4 * H3);               // [nbc + 1] per warp
    unsigned* run = sm_off + nbc + 1;                                       // [H3] per warp
    float* svc = reinterpret_cast<float*>(run + H3);                        // [3][nbc]: v_c of the brick
    float* svn = svc + 3 * nbc;                                             // [3][H3]: v_c* of the halo region
    // the first round's codes and ids first, so their latency overlaps the staging
    int nchi[3] = {0, 0, 0}, nnu[3] = {0, 0, 0};
    float noff[3] = {0.0f, 0.0f, 0.0f};        // 2-byte codes: the next round's decoded offsets
    unsigned nid = 0;
    if (p0 + lane < p1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            nchi[d] = chi_o.get(d, p0 + lane);
            nnu[d] = nu_o.get_nu(d, p0 + lane, lim);
        }
        if (sn.id)
            nid = PID == 4 ? reinterpret_cast<const unsigned*>(so.id)[p0 + lane] : load_pid(so.id, p0 + lane, g.nid);
        if (NV == 2)
#pragma unroll
            for (int d = 0; d < 3; ++d) noff[d] = pb.dec[nnu[d] + lim];
    }
    passB_stage(g, so, ghost, vc_new, brick, lane, 32, sm_off, run, svc, svn);
    __syncwarp();
    int c0 = upper_cell(sm_off, nbc, p0);      // the cell of each round's first particle
    for (unsigned base = p0; base < p1; base += 32) {
        const unsigned i = base + lane;
        const bool act = i < p1;
        const unsigned am = __ballot_sync(0xffffffffu, act);
        // this round's codes; the next round's are requested now
        const int cchi[3] = {nchi[0], nchi[1], nchi[2]}, cnu[3] = {nnu[0], nnu[1], nnu[2]};
        const float coff[3] = {noff[0], noff[1], noff[2]};
        const unsigned cid = nid;
        if (i + 32 < p1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                nchi[d] = chi_o.get(d, i + 32);
                nnu[d] = nu_o.get_nu(d, i + 32, lim);
            }
            if (sn.id)
                nid = PID == 4 ? reinterpret_cast<const unsigned*>(so.id)[i + 32] : load_pid(so.id, i + 32, g.nid);
        }
        int cnext;
        const int lcell = warp_cells(sm_off, nbc, base, c0, &cnext);
        c0 = cnext;
        if (act) {
            const PbParticle q = pb.move(lcell, svc, cchi, cnu, coff);
            const unsigned peers = __match_any_sync(am, q.ei);
            const int leader = __ffs(peers) - 1;
            unsigned start = 0;
            if (lane == leader) start = run[q.ei];
            start = __shfl_sync(peers, start, leader);
            if (lane == leader) run[q.ei] = start + (unsigned)__popc(peers);
            pb.put(q, svn, start + (unsigned)__popc(peers & ((1u << lane) - 1u)), cid, flags);
        }
        if (NV == 2 && i + 32 < p1)                // the next round's offsets, its codes having arrived
#pragma unroll
            for (int d = 0; d < 3; ++d) noff[d] = pb.dec[nnu[d] + lim];
        __syncwarp();
    }
}

// Global sums of the current store (Section 2.3.3's bookkeeping): the
// momenta exactly as cube_decode returns them (v_c + decoded offset, FP32),
// each rounded to a multiple of 2^-24 and summed exactly in int64, so the
// result is independent of the summation order and within N 2^-25 of the
// exact sum of the decoded values; and the particle count as the sum of the
// cell counts.  One CTA per brick, one 64-bit atomic per warp and quantity.
template <int NV>
__global__ void __launch_bounds__(T_BRICK) k_store_sums(Geo g, StoreDev s, const float* __restrict__ dec,
                                                        long long* __restrict__ out4) {
    extern __shared__ unsigned sm_off[];
    const int nbc = g.B * g.B * g.B;
    const int L0 = blockIdx.x * nbc;
    for (int c = threadIdx.x; c <= nbc; c += blockDim.x) sm_off[c] = s.offsets[L0 + c];
    long long cnt = 0;
    for (int c = threadIdx.x; c < nbc; c += blockDim.x) cnt += s.counts[L0 + c];
    __syncthreads();
    const unsigned q1 = min(sm_off[nbc], (unsigned)g.Np);
    long long m[3] = {0, 0, 0};
    for (unsigned i = min(sm_off[0], q1) + threadIdx.x; i < q1; i += blockDim.x) {
        const int lc = upper_cell(sm_off, nbc, i);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int nu = load_nu<NV>(s.nu, d * g.Np + i, g.nulim);
            m[d] += vel_fix(s.vc[(int64_t)d * g.Ncc + L0 + lc] + dec[nu + g.nulim]);
        }
    }
    // warp sums, then the block's in shared memory, then one atomic per sum and block
    __shared__ long long part[4][T_BRICK / 32];
    long long v[4] = {m[0], m[1], m[2], cnt};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane == 0) part[k][wid] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[threadIdx.x][i];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(&out4[threadIdx.x]), (unsigned long long)t);
    }
}

template <int NX, int NV>
struct Disp {
    static void passA(const Geo& g, const StoreDev& s, const float* phig, const CUtensorMap& tmap, int use_tma,
                      const CodecDev& cur, float kick, float dc, const StepScratch& w, const DriftDebug& dbg,
                      size_t sm, cudaStream_t st, const Batch& bt) {
        const dim3 grid(g.nb, g.nb, g.nb * bt.members);
        const bool bat = bt.members > 1 || bt.ms;
        if (g.F == 16) {
            if (bat) k_passA<NX, NV, 16, true><<<grid, PA_T, sm, st>>>(g, s, phig, tmap, use_tma, cur, kick, dc, w, dbg, bt);
            else k_passA<NX, NV, 16, false><<<grid, PA_T, sm, st>>>(g, s, phig, tmap, use_tma, cur, kick, dc, w, dbg, bt);
        } else {
            if (bat) k_passA<NX, NV, 0, true><<<grid, PA_T, sm, st>>>(g, s, phig, tmap, use_tma, cur, kick, dc, w, dbg, bt);
            else k_passA<NX, NV, 0, false><<<grid, PA_T, sm, st>>>(g, s, phig, tmap, use_tma, cur, kick, dc, w, dbg, bt);
        }
    }
    static void passB(const Geo& g, const StoreDev& so, const StoreDev& sn, const CodecDev& cur,
                      const CodecDev& next, float dc, const unsigned* ghost, const float* vcn, unsigned* flags,
                      const int* big, size_t sm, cudaStream_t st, const Batch& bt) {
        // CTAs for crowded bricks first (at most Np / (PB_BIG + 1) of them exist)
        const int nbig_ctas = (int)std::min<int64_t>(2 * g.nsm, g.Np / (PB_BIG + 1));
        const int grid = nbig_ctas + (g.nbricks + PB_WARPS - 1) / PB_WARPS;
        const bool narrow = g.nid == 1 || g.nid == 2;
        if (bt.members > 1 || bt.ms) {
            const dim3 gb(grid, bt.members);
            if (narrow) k_passB<NX, NV, true, 0><<<gb, PB_WARPS * 32, sm, st>>>(g, so, sn, cur, next, dc, ghost, vcn, flags, big, nbig_ctas, bt);
            else k_passB<NX, NV, true, 4><<<gb, PB_WARPS * 32, sm, st>>>(g, so, sn, cur, next, dc, ghost, vcn, flags, big, nbig_ctas, bt);
        } else {
            if (narrow) k_passB<NX, NV, false, 0><<<grid, PB_WARPS * 32, sm, st>>>(g, so, sn, cur, next, dc, ghost, vcn, flags, big, nbig_ctas, bt);
            else k_passB<NX, NV, false, 4><<<grid, PB_WARPS * 32, sm, st>>>(g, so, sn, cur, next, dc, ghost, vcn, flags, big, nbig_ctas, bt);
        }
    }
};

template <int NX, int NV>
void set_smem_attrs() {
    static bool done = false;
    if (done) return;
    const int lim = 200 * 1024;
    cudaFuncSetAttribute(k_passA<NX, NV, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_passA<NX, NV, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_passA<NX, NV, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_passA<NX, NV, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_passB<NX, NV, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_passB<NX, NV, true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_passB<NX, NV, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_passB<NX, NV, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_deposit<NX, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_deposit<NX, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_deposit<NX, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_deposit<NX, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    done = true;
}

// one word of every listed member of a batch set to zero
__global__ void k_zero_slot_words(unsigned* p, Batch bt) {
    for (int i = threadIdx.x; i < bt.members; i += blockDim.x) moved(p, slot_member(bt, i) * bt.stride)[0] = 0u;
}

// every entry of the 2-byte tables as VelTables rebuilds it, against the tables
__global__ void k_check_vel_tables(int lim, CodecDev c, long long* out2) {
    const VelTables vt{c.dec, c.thr, c.vdel, VelApprox{c.est[3], c.est[4], 2 * lim + 1}, lim};
    long long bad = 0, whole = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= lim + 1; k += gridDim.x * blockDim.x) {
        if (k <= lim) {
            bad += __float_as_int(vt.dec(k)) != __float_as_int(c.dec[lim + k]);
            bad += __float_as_int(vt.dec(-k)) != __float_as_int(c.dec[lim - k]);
        }
        bad += __float_as_int(vt.thr(k)) != __float_as_int(c.thr[k]);
        if (k >= 1 && k <= lim) {
            const unsigned b = c.vdel[k];
            whole += (vdelta(b, 0) == -8) + (vdelta(b, 4) == -8);
        }
    }
    block_sum_to(bad, &out2[0]);
    block_sum_to(whole, &out2[1]);
}

// the step's cleared scratch of every stepped member of a batch: the
// fixed-point momentum sums [3][Ncc] and the migration / crowded-brick words
__global__ void k_batch_clear(int64_t n64, long long* __restrict__ vsum, int* __restrict__ mig, Batch bt) {
    if (bt.ms && !bt.ms[blockIdx.y].active) return;
    const int m = slot_member(bt, blockIdx.y);
    vsum = moved(vsum, m * bt.stride);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n64; t += (int64_t)gridDim.x * blockDim.x)
        vsum[t] = 0;
    if (blockIdx.x == 0 && threadIdx.x < 2) moved(mig, m * bt.stride)[threadIdx.x] = 0;
}

}  // namespace

// ------------------------------------------------------------------ launchers
void launch_batch_clear(const Geo& g, long long* vsum, int* maxmig, cudaStream_t st, const Batch& bt) {
    const int64_t n = 3 * (int64_t)g.Ncc;
    k_batch_clear<<<dim3((unsigned)std::min<int64_t>(1024, (n + 255) / 256), bt.members), 256, 0, st>>>(n, vsum,
                                                                                                     maxmig, bt);
}

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

void launch_encode_keys(const Geo& g, const float* pos, const float* vel, unsigned* key, unsigned* val,
                        unsigned* counts, long long* vsum, unsigned* flags, cudaStream_t st) {
    if (g.nchi == 1) k_encode_keys<1><<<nblk(g.Np, 256), 256, 0, st>>>(g, pos, vel, key, val, counts, vsum, flags);
    else k_encode_keys<2><<<nblk(g.Np, 256), 256, 0, st>>>(g, pos, vel, key, val, counts, vsum, flags);
}

void launch_vc_finalize(const Geo& g, const unsigned* counts, const long long* vsum, float* vc, cudaStream_t st) {
    k_vc_finalize<<<nblk(g.Ncc, 256), 256, 0, st>>>(g.Ncc, counts, vsum, vc);
}

int encode_sigma_blocks(const Geo& g) { return (int)std::min<int64_t>(1024, std::max<int64_t>(1, nblk(g.Np, 256))); }

void launch_encode_sigma(const Geo& g, const float* vel, const unsigned* key, const float* vc, float* part,
                         cudaStream_t st) {
    k_encode_sigma<<<encode_sigma_blocks(g), 256, 0, st>>>(g, vel, key, vc, part);
}

void launch_sigma_finalize(const float* part, int nparts, double count, double ratio, double fixed,
                           double* sigma_out, cudaStream_t st, const Batch& bt) {
    k_sigma_finalize<<<bt.members, 1024, 0, st>>>(part, nparts, count, ratio, fixed, sigma_out, bt);
}

void launch_codec_tables(int nulim, const double* tanv, const double* tanh_, const CodecDev& c, cudaStream_t st,
                         const Batch& bt) {
    // 1-byte codes (nulim 127) fit one block, which also builds the bucket table
    const bool one = nulim + 2 <= 256;
    k_codec_tables<<<dim3(nblk(nulim + 2, 256), bt.members), 256, 0, st>>>(nulim, tanv, tanh_, c.sigma, c.dec, c.thr,
                                                                          c.est, one ? c.vtab : nullptr,
                                                                          one ? nullptr : c.vdel, bt);
}

void launch_encode_scatter(const Geo& g, const float* pos, const float* vel, const unsigned* id_in,
                           const unsigned* key_sorted, const unsigned* perm, const float* vc, const CodecDev& c,
                           StoreDev s, cudaStream_t st) {
    int nb = nblk(g.Np, 256);
    if (g.nchi == 1 && g.nnu == 1) k_encode_scatter<1, 1><<<nb, 256, 0, st>>>(g, pos, vel, id_in, key_sorted, perm, vc, c.thr, c.est, s);
    else if (g.nchi == 1) k_encode_scatter<1, 2><<<nb, 256, 0, st>>>(g, pos, vel, id_in, key_sorted, perm, vc, c.thr, c.est, s);
    else if (g.nnu == 1) k_encode_scatter<2, 1><<<nb, 256, 0, st>>>(g, pos, vel, id_in, key_sorted, perm, vc, c.thr, c.est, s);
    else k_encode_scatter<2, 2><<<nb, 256, 0, st>>>(g, pos, vel, id_in, key_sorted, perm, vc, c.thr, c.est, s);
}

void launch_max_speed(const Geo& g, const StoreDev& s, const float* dec, unsigned* vmax_bits, cudaStream_t st,
                      const Batch& bt) {
    size_t sm = (size_t)(g.B * g.B * g.B + 1) * sizeof(unsigned);
    if (bt.members == 1 && !bt.ms) cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned), st);
    else k_zero_slot_words<<<1, 256, 0, st>>>(vmax_bits, bt);
    const dim3 grid(g.nbricks, bt.members);
    if (g.nnu == 1) k_max_speed<1><<<grid, T_BRICK, sm, st>>>(g, s, dec, vmax_bits, bt);
    else k_max_speed<2><<<grid, T_BRICK, sm, st>>>(g, s, dec, vmax_bits, bt);
}

void launch_decode(const Geo& g, const StoreDev& s, const float* dec, float* pos, float* vel, unsigned* id,
                   cudaStream_t st) {
    size_t sm = (size_t)(g.B * g.B * g.B + 1) * sizeof(unsigned);
    if (g.nchi == 1 && g.nnu == 1) k_decode<1, 1><<<g.nbricks, T_BRICK, sm, st>>>(g, s, dec, pos, vel, id);
    else if (g.nchi == 1) k_decode<1, 2><<<g.nbricks, T_BRICK, sm, st>>>(g, s, dec, pos, vel, id);
    else if (g.nnu == 1) k_decode<2, 1><<<g.nbricks, T_BRICK, sm, st>>>(g, s, dec, pos, vel, id);
    else k_decode<2, 2><<<g.nbricks, T_BRICK, sm, st>>>(g, s, dec, pos, vel, id);
}

static size_t deposit_smem(const Geo& g) {
    const int E = g.B + 1, E3 = E * E * E;
    return (size_t)dep_acc_words(g.F) * 4 + (size_t)(3 * E3 + 1) * 4 + DEP_QCAP;
}

void launch_deposit(const Geo& g, const StoreDev& s, float* mesh, double scale, cudaStream_t st, const Batch& bt) {
    size_t sm = deposit_smem(g);
    const bool f16 = g.F == 16, bat = bt.members > 1 || bt.ms;
    const dim3 grid(g.nb, g.nb, g.nb * bt.members);
    const float fs = (float)scale;
    if (g.nchi == 1) {
        set_smem_attrs<1, 1>(); set_smem_attrs<1, 2>();
        if (f16) {
            if (bat) k_deposit<1, 16, true><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
            else k_deposit<1, 16, false><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
        } else {
            if (bat) k_deposit<1, 0, true><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
            else k_deposit<1, 0, false><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
        }
    } else {
        set_smem_attrs<2, 1>(); set_smem_attrs<2, 2>();
        if (f16) {
            if (bat) k_deposit<2, 16, true><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
            else k_deposit<2, 16, false><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
        } else {
            if (bat) k_deposit<2, 0, true><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
            else k_deposit<2, 0, false><<<grid, T_BRICK, sm, st>>>(g, s, mesh, fs, bt);
        }
    }
}

static size_t passA_smem(const Geo& g) {
    const int T = g.F + 5, TS = g.F + 8, H3 = g.Bh * g.Bh * g.Bh, nbc = g.B * g.B * g.B;
    // + 128: the tile is placed on a 128-byte boundary at run time
    size_t sm = (size_t)3 * H3 * 8 + 128 + (size_t)T * T * TS * 4 + (size_t)H3 * 4 + (size_t)(nbc + 1) * 4;
    if (g.nnu == 1) sm += (size_t)(3 * g.nulim + 3) * 4 + VT_N;
    sm += (size_t)3 * nbc * 4 + DEP_QCAP;
    return (sm + 15) & ~(size_t)15;
}

void launch_passA(const Geo& g, const StoreDev& s, const float* phig, const CUtensorMap* tmap, const CodecDev& cur,
                  float kick, float dc, const StepScratch& w, const DriftDebug& dbg, cudaStream_t st,
                  const Batch& bt) {
    size_t sm = passA_smem(g);
    static const CUtensorMap none{};
    const CUtensorMap& tm = tmap ? *tmap : none;
    const int use = tmap != nullptr;
    if (g.nchi == 1 && g.nnu == 1) { set_smem_attrs<1, 1>(); Disp<1, 1>::passA(g, s, phig, tm, use, cur, kick, dc, w, dbg, sm, st, bt); }
    else if (g.nchi == 1) { set_smem_attrs<1, 2>(); Disp<1, 2>::passA(g, s, phig, tm, use, cur, kick, dc, w, dbg, sm, st, bt); }
    else if (g.nnu == 1) { set_smem_attrs<2, 1>(); Disp<2, 1>::passA(g, s, phig, tm, use, cur, kick, dc, w, dbg, sm, st, bt); }
    else { set_smem_attrs<2, 2>(); Disp<2, 2>::passA(g, s, phig, tm, use, cur, kick, dc, w, dbg, sm, st, bt); }
}

void launch_cells(const Geo& g, const StepScratch& w, unsigned* off_new, float* vc_new, cudaStream_t st,
                  const Batch& bt) {
    if (bt.members > 1 || bt.ms) k_cells<true><<<dim3(nblk(g.Ncc, 256), bt.members), 256, 0, st>>>(g, w, off_new, vc_new, bt);
    else k_cells<false><<<nblk(g.Ncc, 256), 256, 0, st>>>(g, w, off_new, vc_new, bt);
}

static size_t passB_smem(const Geo& g) {
    const int H3 = g.Bh * g.Bh * g.Bh, nbc = g.B * g.B * g.B;
    size_t sm = (size_t)PB_WARPS * (4 * nbc + 1 + 4 * H3) * 4;
    if (g.nnu == 1) sm += (size_t)(3 * g.nulim + 3) * 4 + VT_N;
    return (sm + 15) & ~(size_t)15;
}

void launch_passB(const Geo& g, const StoreDev& so, const StoreDev& sn, const CodecDev& cur, const CodecDev& next,
                  float dc, const StepScratch& w, cudaStream_t st, const Batch& bt) {
    size_t sm = passB_smem(g);
    const float* vcn = sn.vc;
    if (g.nchi == 1 && g.nnu == 1) { set_smem_attrs<1, 1>(); Disp<1, 1>::passB(g, so, sn, cur, next, dc, w.ghost, vcn, w.flags, w.big, sm, st, bt); }
    else if (g.nchi == 1) { set_smem_attrs<1, 2>(); Disp<1, 2>::passB(g, so, sn, cur, next, dc, w.ghost, vcn, w.flags, w.big, sm, st, bt); }
    else if (g.nnu == 1) { set_smem_attrs<2, 1>(); Disp<2, 1>::passB(g, so, sn, cur, next, dc, w.ghost, vcn, w.flags, w.big, sm, st, bt); }
    else { set_smem_attrs<2, 2>(); Disp<2, 2>::passB(g, so, sn, cur, next, dc, w.ghost, vcn, w.flags, w.big, sm, st, bt); }
}

void launch_check_vel_tables(int lim, const CodecDev& c, long long* out2, cudaStream_t st) {
    cudaMemsetAsync(out2, 0, 2 * sizeof(long long), st);
    k_check_vel_tables<<<nblk(lim + 2, 256), 256, 0, st>>>(lim, c, out2);
}

void launch_store_sums(const Geo& g, const StoreDev& s, const float* dec, long long* out4, cudaStream_t st) {
    size_t sm = (size_t)(g.B * g.B * g.B + 1) * sizeof(unsigned);
    cudaMemsetAsync(out4, 0, 4 * sizeof(long long), st);
    if (g.nnu == 1) k_store_sums<1><<<g.nbricks, T_BRICK, sm, st>>>(g, s, dec, out4);
    else k_store_sums<2><<<g.nbricks, T_BRICK, sm, st>>>(g, s, dec, out4);
}

}  // namespace cube
