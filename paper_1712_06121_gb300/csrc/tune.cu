// Autotuner of the storage-order brick: the tile shape of the deposit, of
// pass A's potential tile and of pass B's re-sort.  Every brick side gives
// bit-identical results (integer CIC weights, stable per-cell order), so the
// choice affects speed only.  Small meshes favour small bricks (more CTAs,
// smaller tiles), large meshes the largest.
#include <string>
#include <vector>

#include "cube.h"
#include "kernels.h"

namespace cube {
cube_status served_fail(cube_status s, const char* msg);
}

extern "C" cube_status cube_autotune_brick(const cube_params* params, const float* pos, const float* vel,
                                           double a, double sigma, int32_t n_steps, void* cuda_stream,
                                           int32_t* best_brick, double* ms_per_step) {
    using cube::served_fail;
    if (!params || !pos || !vel || !best_brick) return served_fail(CUBE_E_ARG, "NULL argument");
    if (n_steps < 1 || n_steps > 100) return served_fail(CUBE_E_ARG, "n_steps in [1, 100]");
    if (!(a > 0.0)) return served_fail(CUBE_E_ARG, "a must be > 0");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int cand[3] = {1, 2, 4};
    double best = 0.0;
    *best_brick = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return served_fail(CUBE_E_CUDA, "event creation");
    cube_status out = CUBE_OK;
    for (int i = 0; i < 3; ++i) {
        if (ms_per_step) ms_per_step[i] = -1.0;
        cube_params p = *params;
        p.brick = cand[i];
        cube_ctx* c = nullptr;
        if (cube_create(&p, st, &c) != CUBE_OK) continue;         // brick not valid for this mesh
        // one untimed step (module loading, caches), then n_steps timed ones;
        // small steps in a keep every particle in place
        cube_status s = cube_encode(c, pos, vel, nullptr, a, sigma);
        double t = a;
        const double da = 1e-4 * a;
        if (s == CUBE_OK) s = cube_pm_step(c, t, t + da);
        t += da;
        float ms = 0.0f;
        if (s == CUBE_OK) {
            cudaEventRecord(e0, st);
            for (int k = 0; k < n_steps && s == CUBE_OK; ++k, t += da) s = cube_pm_step(c, t, t + da);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        cube_destroy(c);
        if (s != CUBE_OK) {
            out = s;
            break;
        }
        const double per = (double)ms / n_steps;
        if (ms_per_step) ms_per_step[i] = per;
        if (*best_brick == 0 || per < best) {
            best = per;
            *best_brick = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out == CUBE_OK && *best_brick == 0) return served_fail(CUBE_E_ARG, "no valid brick size");
    return out;
}
