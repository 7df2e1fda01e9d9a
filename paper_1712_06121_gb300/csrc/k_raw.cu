// Uncompressed FP32 particles: the same PM step on plain float positions and
// momenta (no codes, no cell order), the comparison arm of the precision
// study of Section 3 (the paper compares its compressed runs with an
// uncompressed PM code).  One thread per particle.
//   deposit    CIC mass of each particle onto the fine mesh (float atomics;
//              the summation order, and so the last bit, is not fixed)
//   kick/drift CIC gather of the FD4 gradient of Phi (ghosted copy), kick,
//              drift, periodic wrap
#include "kernels.h"

namespace cube {

namespace {

constexpr int RAW_T = 256;

// periodic image of x in [0, n); non-finite x gives 0 and sets *bad
__device__ __forceinline__ float wrap_pos(float x, float n, bool* bad) {
    if (!isfinite(x)) {
        *bad = true;
        return 0.0f;
    }
    x -= n * floorf(x / n);
    x -= x >= n ? n : 0.0f;
    return x < 0.0f ? 0.0f : x;
}

// node of x, always inside [0, n - 1] (whatever x holds)
__device__ __forceinline__ int node_of(float x, int n) { return min(max((int)floorf(x), 0), n - 1); }

__global__ void __launch_bounds__(RAW_T) k_raw_encode(int64_t np, float n, const float* __restrict__ pos,
                                                      const float* __restrict__ vel,
                                                      const unsigned* __restrict__ id_in, float* __restrict__ P,
                                                      float* __restrict__ V, unsigned* __restrict__ I,
                                                      unsigned* flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float x = pos[d * np + i], v = vel[d * np + i];
        if (!isfinite(x) || !isfinite(v)) {
            bad = true;
            x = 0.0f;
            v = 0.0f;
        }
        P[d * np + i] = wrap_pos(x, n, &bad);
        V[d * np + i] = v;
    }
    if (I) I[i] = id_in ? id_in[i] : (unsigned)i;
    if (bad) atomicOr(flags, ERR_NONFINITE);
}

__global__ void __launch_bounds__(RAW_T) k_raw_deposit(Geo g, const float* __restrict__ P, float* __restrict__ mesh,
                                                       float mass) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Np) return;
    int n0[3], n1[3];
    float w1[3], w0[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float x = P[d * g.Np + i];
        const int c = node_of(x, g.N);
        w1[d] = x - (float)c;
        w0[d] = 1.0f - w1[d];
        n0[d] = c;
        n1[d] = c + 1 == g.N ? 0 : c + 1;
    }
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const float w = mass * (dz ? w1[2] : w0[2]) * (dy ? w1[1] : w0[1]) * (dx ? w1[0] : w0[0]);
                atomicAdd(&mesh[((int64_t)(dz ? n1[2] : n0[2]) * g.N + (dy ? n1[1] : n0[1])) * g.S +
                                (dx ? n1[0] : n0[0])],
                          w);
            }
}

// FD4 gradient along one axis, interpolated between nodes c and c + 1:
// (1 - w) G(c) + w G(c + 1), G(m) = 8 (phi[m+1] - phi[m-1]) - (phi[m+2] - phi[m-2]),
// phi[k] = r[k + 2] for k = -2 .. 3
__device__ __forceinline__ float fd4_line(const float* r, float w) {
    const float g0 = 8.0f * (r[3] - r[1]) - (r[4] - r[0]);
    const float g1 = 8.0f * (r[4] - r[2]) - (r[5] - r[1]);
    return (1.0f - w) * g0 + w * g1;
}

__global__ void __launch_bounds__(RAW_T) k_raw_kick_drift(Geo g, float* __restrict__ P, float* __restrict__ V,
                                                          const float* __restrict__ phig, float kick, float drift,
                                                          unsigned* flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Np) return;
    float x[3], w[3];
    int k[3][6];                                     // periodic node coordinates c - 2 .. c + 3
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        x[d] = P[d * g.Np + i];
        const int c = node_of(x[d], g.N);
        w[d] = x[d] - (float)c;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            int q = c - 2 + m;
            q += q < 0 ? g.N : 0;
            q -= q >= g.N ? g.N : 0;
            k[d][m] = q;
        }
    }
    auto at = [&](int ix, int iy, int iz) { return __ldg(&phig[phig_index(g.N, k[0][ix], k[1][iy], k[2][iz])]); };
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            float r[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) r[m] = at(m, 2 + a, 2 + b);
            gx += (a ? w[1] : 1.0f - w[1]) * (b ? w[2] : 1.0f - w[2]) * fd4_line(r, w[0]);
#pragma unroll
            for (int m = 0; m < 6; ++m) r[m] = at(2 + a, m, 2 + b);
            gy += (a ? w[0] : 1.0f - w[0]) * (b ? w[2] : 1.0f - w[2]) * fd4_line(r, w[1]);
#pragma unroll
            for (int m = 0; m < 6; ++m) r[m] = at(2 + a, 2 + b, m);
            gz += (a ? w[0] : 1.0f - w[0]) * (b ? w[1] : 1.0f - w[1]) * fd4_line(r, w[2]);
        }
    const float fsc = -1.0f / 12.0f;
    const float f[3] = {gx * fsc, gy * fsc, gz * fsc};
    const float n = (float)g.N;
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float v = __fmaf_rn(f[d], kick, V[d * g.Np + i]);
        V[d * g.Np + i] = v;
        P[d * g.Np + i] = wrap_pos(__fmaf_rn(v, drift, x[d]), n, &bad);
    }
    if (bad) atomicOr(flags, ERR_NONFINITE);
}

// sum of the momenta in 2^-24 fixed point (exact, any order)
__global__ void __launch_bounds__(RAW_T) k_raw_momentum(int64_t np, const float* __restrict__ V, long long* out3) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int d = 0; d < 3; ++d) block_sum_to(i < np ? vel_fix(V[d * np + i]) : 0, &out3[d]);
}

// largest |p| over particles and axes, as the bits of a non-negative float
__global__ void __launch_bounds__(RAW_T) k_raw_max_speed(int64_t np, const float* __restrict__ V,
                                                         unsigned* __restrict__ vmax_bits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.0f;
    if (i < np) m = fmaxf(fmaxf(fabsf(V[i]), fabsf(V[np + i])), fabsf(V[2 * np + i]));
    block_max_to(__float_as_uint(m), vmax_bits);
}

__global__ void k_iota(unsigned* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (unsigned)i;
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + RAW_T - 1) / RAW_T); }

}  // namespace

void launch_raw_encode(const Geo& g, const float* pos, const float* vel, const unsigned* id_in, float* P, float* V,
                       unsigned* I, unsigned* flags, cudaStream_t st) {
    k_raw_encode<<<nblk(g.Np), RAW_T, 0, st>>>(g.Np, (float)g.N, pos, vel, id_in, P, V, I, flags);
}

void launch_raw_deposit(const Geo& g, const float* P, float* mesh, float mass, cudaStream_t st) {
    k_raw_deposit<<<nblk(g.Np), RAW_T, 0, st>>>(g, P, mesh, mass);
}

void launch_raw_kick_drift(const Geo& g, float* P, float* V, const float* phig, float kick, float drift,
                           unsigned* flags, cudaStream_t st) {
    k_raw_kick_drift<<<nblk(g.Np), RAW_T, 0, st>>>(g, P, V, phig, kick, drift, flags);
}

void launch_iota(unsigned* out, int64_t n, cudaStream_t st) { k_iota<<<nblk(n), RAW_T, 0, st>>>(out, n); }

void launch_raw_max_speed(const Geo& g, const float* V, unsigned* vmax_bits, cudaStream_t st) {
    cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned), st);
    k_raw_max_speed<<<nblk(g.Np), RAW_T, 0, st>>>(g.Np, V, vmax_bits);
}

void launch_raw_momentum(const Geo& g, const float* V, long long* out3, cudaStream_t st) {
    cudaMemsetAsync(out3, 0, 3 * sizeof(long long), st);
    k_raw_momentum<<<nblk(g.Np), RAW_T, 0, st>>>(g.Np, V, out3);
}

}  // namespace cube
