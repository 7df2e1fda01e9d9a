// Internal launch interface between libcube's host code and its kernels.
#pragma once

#include <string>
#include <type_traits>

#include <cuda.h>

#include "cube_common.cuh"

namespace cube {

// Stable ranking of one round of blockDim.x items by `digit` in [0, nd),
// nd <= 256:
// items are ordered by (warp, lane), i.e. by thread index, and equal digits
// keep that order.  run[nd] holds each digit's next free position and is
// advanced by the round's counts; wcnt[NWARPS * nd] is scratch.  Every thread
// of the block must call it (it synchronises).  Returns the item's position,
// or -1 for inactive threads.
template <int NWARPS>
__device__ __forceinline__ int stable_round_rank(int digit, bool active, unsigned* run, unsigned* wcnt, int nd) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NWARPS * nd; i += blockDim.x) wcnt[i] = 0u;
    __syncthreads();
    unsigned act = __ballot_sync(0xffffffffu, active);
    int lrank = 0;
    if (active) {
        unsigned peers = same_value_lanes(act, digit);
        lrank = __popc(peers & ((1u << lane) - 1u));
        if (lrank == 0) wcnt[w * nd + digit] = (unsigned)__popc(peers);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        unsigned s = run[d];
        for (int ww = 0; ww < NWARPS; ++ww) {
            unsigned t = wcnt[ww * nd + d];
            wcnt[ww * nd + d] = s;
            s += t;
        }
        run[d] = s;
    }
    __syncthreads();
    int pos = active ? (int)(wcnt[w * nd + digit] + (unsigned)lrank) : -1;
    __syncthreads();
    return pos;
}

// ------------------------------------------------------------ batches
// A batched launch steps several members (simulations with the same
// geometry) at once: member m's device buffers are member 0's plus m * stride
// bytes, so every kernel of the step takes one extra grid dimension over the
// members and moves its pointers by m * stride.  A single context is the
// batch of one (members 1, stride 0, no per-member table).
struct MemberStep {
    float kick, dc;     // the step's kick factor and drift per coarse cell
    double ratio;       // momentum growth ratio of the codec-scale update
    int active;         // 0: the slot steps nothing (its kernels return at once)
    int member;         // the member this grid slot steps
};
// A launch's grid has one slot per listed member: with a per-member table,
// slot i steps member ms[i].member (a batch step lists only the members it
// moves, so members that sit it out cost no CTAs); without one, slot i is
// member i.  host_members mirrors ms[i].member for launches issued member by
// member from the host (null: slot i is member i).
struct Batch {
    int members;                 // slots of the launch
    size_t stride;               // bytes between consecutive members' buffers
    const MemberStep* ms;        // [members] (device) or null
    const int* host_members;     // [members] (host) or null
};
__host__ __device__ __forceinline__ int slot_member(const Batch& bt, int slot) {
#ifdef __CUDA_ARCH__
    return bt.ms ? bt.ms[slot].member : slot;
#else
    return bt.host_members ? bt.host_members[slot] : slot;
#endif
}
template <class T>
__host__ __device__ __forceinline__ T* moved(T* p, size_t off) {
    return p ? reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<typename std::remove_const<T>::type*>(p)) + off)
             : p;
}

// ------------------------------------------------------------ cube_api.cu
void set_last_error(const std::string& msg);     // message for cube_last_error()

// ------------------------------------------------------------ k_scan.cu
int scan_tmp_words(int64_t n);
void exclusive_scan(const unsigned* in, unsigned* out, int64_t n, unsigned* tmp, cudaStream_t st,
                    const Batch& bt = Batch{1, 0, nullptr, nullptr});
// out2[0] = 64-bit sum, out2[1] = maximum of n counts
void count_totals(const unsigned* counts, int64_t n, unsigned long long* out2, cudaStream_t st);
int64_t radix_tmp_words(int64_t n);
void radix_sort_pairs(unsigned* keys, unsigned* vals, int64_t n, int key_bits, unsigned* tmp, cudaStream_t st);

// ------------------------------------------------------------ k_store.cu
struct StoreDev {
    unsigned* counts;   // [Ncc]
    unsigned* offsets;  // [Ncc + 1]
    float* vc;          // [3][Ncc]
    void* chi;          // [3][Np]
    void* nu;           // [3][Np]
    void* id;           // [Np] particle IDs of Geo::nid bytes (1, 2 or 4), or null
};

struct CodecDev {
    float* dec;         // [2 lim + 1]: dec[nu + lim] = tan(pi nu / M) * sqrt(2 sigma^2 / pi)
    float* thr;         // [lim + 2]: encode thresholds (see nu_from_thresholds)
    float* est;         // [8]: s and M/pi for the starting guess; [2] the first bucket key of vtab (int bits);
                        // [3], [4]: pi / (2M) and 1 / s of the 2-byte tables' approximation (VelApprox)
    unsigned char* vtab;   // [VT_N] (1-byte codes): code at the start of each bucket of |d| (see nu_from_table)
    double* sigma;      // device scalar
    unsigned char* vdel;   // [lim + 2] (2-byte codes): corrections of dec and thr to tan_half_steps (VelTables)
};

struct DriftDebug {
    int* cell_old;      // [3][Np] or null
    float* u_new;       // [3][Np]
    float* p;           // [3][Np]
    float* force;       // [3][Np]: gathered -grad Phi before the kick
};

struct StepScratch {
    unsigned* counts_new;   // [Ncc]
    long long* vsum_new;    // [3][Ncc]
    unsigned* ghost;        // [nbricks * Bh^3 + 1]: per-brick histograms in flattened
                            // (cell, brick) order, scanned in place into starts
    float* part;            // [max(nbricks, blocks)] partial sums
    unsigned* flags;        // device error flags
    int* maxmig;            // largest |cell shift| of the step
    int* big;               // [1 + nbricks]: number of bricks with more than PB_BIG
                            // particles, then their indices (listed by pass A)
};

// the same buffers of the member `off` bytes further on
__host__ __device__ __forceinline__ StoreDev moved(const StoreDev& s, size_t off) {
    return StoreDev{moved(s.counts, off), moved(s.offsets, off), moved(s.vc, off), moved(s.chi, off),
                    moved(s.nu, off), moved(s.id, off)};
}
__host__ __device__ __forceinline__ CodecDev moved(const CodecDev& c, size_t off) {
    return CodecDev{moved(c.dec, off), moved(c.thr, off), moved(c.est, off), moved(c.vtab, off), moved(c.sigma, off),
                    moved(c.vdel, off)};
}
__host__ __device__ __forceinline__ StepScratch moved(const StepScratch& w, size_t off) {
    return StepScratch{moved(w.counts_new, off), moved(w.vsum_new, off), moved(w.ghost, off), moved(w.part, off),
                       moved(w.flags, off), moved(w.maxmig, off), moved(w.big, off)};
}
// a batch of one: a single context's launch
constexpr Batch kSingle{1, 0, nullptr, nullptr};

void launch_encode_keys(const Geo& g, const float* pos, const float* vel, unsigned* key, unsigned* val,
                        unsigned* counts, long long* vsum, unsigned* flags, cudaStream_t st);
void launch_vc_finalize(const Geo& g, const unsigned* counts, const long long* vsum, float* vc, cudaStream_t st);
int encode_sigma_blocks(const Geo& g);
void launch_encode_sigma(const Geo& g, const float* vel, const unsigned* key_sorted_or_raw, const float* vc,
                         float* part, cudaStream_t st);
void launch_sigma_finalize(const float* part, int nparts, double count, double ratio, double fixed,
                           double* sigma_out, cudaStream_t st, const Batch& bt = Batch{1, 0, nullptr, nullptr});
void launch_codec_tables(int nulim, const double* tanv, const double* tanh, const CodecDev& c, cudaStream_t st,
                         const Batch& bt = Batch{1, 0, nullptr, nullptr});
void launch_encode_scatter(const Geo& g, const float* pos, const float* vel, const unsigned* id_in,
                           const unsigned* key_sorted, const unsigned* perm, const float* vc, const CodecDev& c,
                           StoreDev s, cudaStream_t st);
void launch_decode(const Geo& g, const StoreDev& s, const float* dec, float* pos, float* vel, unsigned* id,
                   cudaStream_t st);
void launch_deposit(const Geo& g, const StoreDev& s, float* mesh, double scale, cudaStream_t st,
                    const Batch& bt = Batch{1, 0, nullptr, nullptr});
// phig: ghosted Phi; tmap: TMA map of phig with the brick's tile as its box, or NULL (cp.async loads)
// (tmap: a 4-D map over (x, y, z, member) of the members' ghosted Phi)
void launch_passA(const Geo& g, const StoreDev& s, const float* phig, const CUtensorMap* tmap, const CodecDev& cur,
                  float kick, float dc, const StepScratch& w, const DriftDebug& dbg, cudaStream_t st,
                  const Batch& bt = Batch{1, 0, nullptr, nullptr});
// a batch step's cleared scratch (momentum sums, migration words) of its stepped members
void launch_batch_clear(const Geo& g, long long* vsum, int* maxmig, cudaStream_t st, const Batch& bt);
void launch_cells(const Geo& g, const StepScratch& w, unsigned* off_new, float* vc_new, cudaStream_t st,
                  const Batch& bt = Batch{1, 0, nullptr, nullptr});
void launch_passB(const Geo& g, const StoreDev& s_old, const StoreDev& s_new, const CodecDev& cur,
                  const CodecDev& next, float dc, const StepScratch& w, cudaStream_t st,
                  const Batch& bt = Batch{1, 0, nullptr, nullptr});
// sums over the current store: out[0..2] momentum of the decoded particles in
// 2^-24 fixed point, out[3] the particle count (sum of the cell counts)
void launch_store_sums(const Geo& g, const StoreDev& s, const float* dec, long long* out4, cudaStream_t st);
// 2-byte codes: out2[0] entries of dec / thr that VelTables rebuilds differently, out2[1] entries it reads whole
void launch_check_vel_tables(int lim, const CodecDev& c, long long* out2, cudaStream_t st);

// uncompressed FP32 particles (k_raw.cu)
void launch_raw_encode(const Geo& g, const float* pos, const float* vel, const unsigned* id_in, float* P, float* V,
                       unsigned* I, unsigned* flags, cudaStream_t st);
void launch_raw_deposit(const Geo& g, const float* P, float* mesh, float mass, cudaStream_t st);
void launch_raw_kick_drift(const Geo& g, float* P, float* V, const float* phi, float kick, float drift,
                           unsigned* flags, cudaStream_t st);
void launch_raw_momentum(const Geo& g, const float* V, long long* out3, cudaStream_t st);
void launch_iota(unsigned* out, int64_t n, cudaStream_t st);
void launch_raw_max_speed(const Geo& g, const float* V, unsigned* vmax_bits, cudaStream_t st);
// largest |p| of the store (float bits), of every listed member of a batch
void launch_max_speed(const Geo& g, const StoreDev& s, const float* dec, unsigned* vmax_bits, cudaStream_t st,
                      const Batch& bt = Batch{1, 0, nullptr, nullptr});

// ------------------------------------------------------------ k_fft.cu
struct FftPlan {
    int N;              // transform length along every axis
    float2* tw;         // [N] e^{-2 pi i k / N}
    float* k2;          // [N] (2 pi f / N)^2, f the signed frequency of index i
    float* wdec;        // [N] sinc(pi f / N)^(-2 p)  (deconvolution factor per axis)
    double* wpk;        // [N] sinc(pi f / N)^(-4)    (P(k) window correction per axis)
};

bool fft_size_supported(int N);                                                    // compiled mesh sizes
void fft_x_r2c(const FftPlan& p, float* mesh, int S, cudaStream_t st,
               const Batch& bt = Batch{1, 0, nullptr, nullptr});                                      // rows: r2c
void fft_y(const FftPlan& p, float* mesh, int S, bool inverse, cudaStream_t st,
           const Batch& bt = Batch{1, 0, nullptr, nullptr});                                          // y columns
void fft_z(const FftPlan& p, float* mesh, int S, float g0, bool green, cudaStream_t st,
           const Batch& bt = Batch{1, 0, nullptr, nullptr});                                          // z (+ Green, inverse)
void fft_x_c2r(const FftPlan& p, float* mesh, int S, float* phig, cudaStream_t st,
               const Batch& bt = Batch{1, 0, nullptr, nullptr});                                      // rows: c2r into ghosted Phi
int pk_blocks(int N);
void launch_pk_bin(const FftPlan& p, const float* mesh, int S, int nbins, double pfac, double kfund,
                   double* part, cudaStream_t st);
void launch_pk_reduce(const double* part, int nblocks, int nbins, double* k, double* pk, double* nm,
                      cudaStream_t st);
void launch_unpad(const float* mesh, int N, int S, float* out, cudaStream_t st);
// largest |component| of the FD4 gradient / 12 of the ghosted potential over
// all mesh nodes (float bits): an upper bound of every particle's force
// component, which the gather interpolates from these values with CIC weights
void launch_grad_max(const float* phig, int N, unsigned* out_bits, cudaStream_t st);
void launch_unpad_phig(const float* phig, int N, float* out, cudaStream_t st);

}  // namespace cube
