// Device-wide exclusive scan and a stable LSD radix sort (the counting sorts
// that keep the store cell-ordered, Sections 2.1 and 2.3.3).
#include "kernels.h"

namespace cube {

namespace {

constexpr int SCAN_T = 1024;           // threads per scan block
constexpr int SCAN_ITEMS = 4;          // items per thread
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

// inclusive scan of one value per thread over the block; returns the
// inclusive prefix, writes the block total to *total
__device__ unsigned block_inclusive_scan(unsigned v, unsigned* smem_warp, unsigned* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) smem_warp[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned s = lane < nw ? smem_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) smem_warp[lane] = s;
    }
    __syncthreads();
    unsigned add = w > 0 ? smem_warp[w - 1] : 0u;
    unsigned tot = smem_warp[nw - 1];
    __syncthreads();
    *total = tot;
    return v + add;
}

// SCAN_ITEMS = 4 consecutive items of one thread, as one 16-byte load when
// the array is 16-byte aligned and the four items exist
__device__ __forceinline__ void load4(const unsigned* __restrict__ in, int64_t base, int64_t n, bool vec,
                                      unsigned* v) {
    if (vec && base + 3 < n) {
        const uint4 q = *reinterpret_cast<const uint4*>(in + base);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = base + i < n ? in[base + i] : 0u;
    }
}

// (member blockIdx.y of a batch: its arrays are `stride` bytes further on)
__global__ void k_scan_reduce(const unsigned* __restrict__ in, int64_t n, unsigned* __restrict__ bsum, bool vec,
                              Batch bt) {
    __shared__ unsigned sw[32];
    if (bt.ms && !bt.ms[blockIdx.y].active) return;
    const int m = slot_member(bt, blockIdx.y);
    in = moved(in, m * bt.stride);
    bsum = moved(bsum, m * bt.stride);
    unsigned v[SCAN_ITEMS];
    load4(in, (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS, n, vec, v);
    const unsigned s = v[0] + v[1] + v[2] + v[3];
    unsigned tot;
    block_inclusive_scan(s, sw, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// exclusive scan of the block sums in place (single block, any count)
__global__ void k_scan_bsums(unsigned* bsum, int nb, unsigned* total_out, Batch bt) {
    __shared__ unsigned sw[32];
    if (bt.ms && !bt.ms[blockIdx.x].active) return;
    const int m = slot_member(bt, blockIdx.x);
    bsum = moved(bsum, m * bt.stride);
    total_out = moved(total_out, m * bt.stride);
    unsigned carry = 0;
    for (int base = 0; base < nb; base += SCAN_T) {
        int i = base + threadIdx.x;
        unsigned v = i < nb ? bsum[i] : 0u;
        unsigned tot;
        unsigned inc = block_inclusive_scan(v, sw, &tot);
        if (i < nb) bsum[i] = carry + inc - v;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_down(const unsigned* in, int64_t n, const unsigned* __restrict__ bsum, unsigned* out,
                            bool vec, Batch bt) {
    __shared__ unsigned sw[32];
    if (bt.ms && !bt.ms[blockIdx.y].active) return;
    const int m = slot_member(bt, blockIdx.y);
    in = moved(in, m * bt.stride);
    bsum = moved(bsum, m * bt.stride);
    out = moved(out, m * bt.stride);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS];
    load4(in, base, n, vec, v);
    const unsigned s = v[0] + v[1] + v[2] + v[3];
    unsigned tot;
    const unsigned inc = block_inclusive_scan(s, sw, &tot);
    unsigned e[SCAN_ITEMS];
    e[0] = bsum[blockIdx.x] + inc - s;
#pragma unroll
    for (int i = 1; i < SCAN_ITEMS; ++i) e[i] = e[i - 1] + v[i - 1];
    if (vec && base + 3 < n) {
        *reinterpret_cast<uint4*>(out + base) = make_uint4(e[0], e[1], e[2], e[3]);
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i)
            if (base + i < n) out[base + i] = e[i];
    }
}

__global__ void k_write_total(unsigned* out, int64_t n, const unsigned* total, Batch bt) {
    if (bt.ms && !bt.ms[blockIdx.x].active) return;
    const int m = slot_member(bt, blockIdx.x);
    moved(out, m * bt.stride)[n] = *moved(total, m * bt.stride);
}

// 64-bit sum and maximum of n 32-bit counts: out2[0] += sum, out2[1] = max(out2[1], max)
__global__ void k_count_totals(const unsigned* __restrict__ c, int64_t n, unsigned long long* out2) {
    unsigned long long s = 0;
    unsigned m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        s += c[i];
        m = max(m, c[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out2[0], s);
        atomicMax(&out2[1], (unsigned long long)m);
    }
}

// ------------------------------------------------------------ radix sort
constexpr int RX_T = 256;
constexpr int RX_ITEMS = 8;
constexpr int RX_TILE = RX_T * RX_ITEMS;

__global__ void k_radix_hist(const unsigned* __restrict__ keys, int64_t n, int shift, int ntiles,
                             unsigned* __restrict__ hist) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RX_TILE;
    for (int i = 0; i < RX_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * RX_T + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RX_T) k_radix_scatter(const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
                                                        int64_t n, int shift, int ntiles,
                                                        const unsigned* __restrict__ hscan,
                                                        unsigned* __restrict__ kout, unsigned* __restrict__ vout) {
    __shared__ unsigned run[256];
    __shared__ unsigned wcnt[(RX_T / 32) * 256];
    run[threadIdx.x] = hscan[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RX_TILE;
    for (int i = 0; i < RX_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * RX_T + threadIdx.x;
        bool act = idx < n;
        unsigned k = act ? kin[idx] : 0u;
        unsigned v = act ? vin[idx] : 0u;
        int d = (int)((k >> shift) & 255u);
        int pos = stable_round_rank<RX_T / 32>(d, act, run, wcnt, 256);
        if (act && pos >= 0 && pos < n) {
            kout[pos] = k;
            vout[pos] = v;
        }
    }
}

}  // namespace

int scan_tmp_words(int64_t n) { return (int)((n + SCAN_TILE - 1) / SCAN_TILE) + 1; }

void exclusive_scan(const unsigned* in, unsigned* out, int64_t n, unsigned* tmp, cudaStream_t st, const Batch& bt) {
    int nb = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    if (nb == 0) nb = 1;
    unsigned* total = tmp + nb;
    // (members are whole multiples of 256 bytes apart: the same alignment)
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    k_scan_reduce<<<dim3(nb, bt.members), SCAN_T, 0, st>>>(in, n, tmp, vec, bt);
    k_scan_bsums<<<bt.members, SCAN_T, 0, st>>>(tmp, nb, total, bt);
    k_scan_down<<<dim3(nb, bt.members), SCAN_T, 0, st>>>(in, n, tmp, out, vec, bt);
    k_write_total<<<bt.members, 1, 0, st>>>(out, n, total, bt);
}

void count_totals(const unsigned* counts, int64_t n, unsigned long long* out2, cudaStream_t st) {
    cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), st);
    const int64_t nb = (n + 255) / 256;
    k_count_totals<<<(int)(nb < 1024 ? (nb < 1 ? 1 : nb) : 1024), 256, 0, st>>>(counts, n, out2);
}

int64_t radix_tmp_words(int64_t n) {
    int64_t ntiles = (n + RX_TILE - 1) / RX_TILE;
    if (ntiles == 0) ntiles = 1;
    int64_t h = 256 * ntiles;
    return 2 * h + 1 + scan_tmp_words(h) + 2 * n;
}

void radix_sort_pairs(unsigned* keys, unsigned* vals, int64_t n, int key_bits, unsigned* tmp, cudaStream_t st) {
    int ntiles = (int)((n + RX_TILE - 1) / RX_TILE);
    if (ntiles == 0) return;
    int64_t h = 256LL * ntiles;
    unsigned* hist = tmp;
    unsigned* hscan = hist + h;          // h + 1 entries (total at the end)
    unsigned* stmp = hscan + h + 1;
    unsigned* kalt = stmp + scan_tmp_words(h);
    unsigned* valt = kalt + n;
    unsigned *ka = keys, *va = vals, *kb = kalt, *vb = valt;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix_hist<<<ntiles, RX_T, 0, st>>>(ka, n, shift, ntiles, hist);
        exclusive_scan(hist, hscan, h, stmp, st);
        k_radix_scatter<<<ntiles, RX_T, 0, st>>>(ka, va, n, shift, ntiles, hscan, kb, vb);
        unsigned* t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (ka != keys) {
        cudaMemcpyAsync(keys, ka, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, va, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    }
}

}  // namespace cube
