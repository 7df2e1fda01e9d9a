// libcube C ABI: context, tables, and the order of kernels of each call.
// See include/cube.h for the contract of every entry point.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "cube.h"
#include "kernels.h"

using namespace cube;

namespace {

thread_local std::string g_err;

cube_status fail(cube_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? CUBE_E_NOMEM : CUBE_E_CUDA,     \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

constexpr double PI = 3.141592653589793;

// ---------------------------------------------------------------- host FP64 cosmology
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
struct Gauss {
    std::vector<double> x, w;
    explicit Gauss(int n) : x(n), w(n) {
        for (int i = 0; i < n; ++i) {
            double z = std::cos(PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
            for (int it = 0; it < 100; ++it) {
                double p1 = 1.0, p2 = 0.0;
                for (int j = 1; j <= n; ++j) {
                    double p3 = p2;
                    p2 = p1;
                    p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
                }
                pp = n * (z * p1 - p2) / (z * z - 1.0);
                double dz = p1 / pp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
        }
    }
};

const Gauss& gauss64() {
    static Gauss g(64);
    return g;
}

template <class Fn>
double integrate(Fn f, double a0, double a1, int panels = 16) {
    const Gauss& g = gauss64();
    double s = 0.0, h = (a1 - a0) / panels;
    for (int p = 0; p < panels; ++p) {
        double lo = a0 + p * h, mid = lo + 0.5 * h;
        for (size_t i = 0; i < g.x.size(); ++i) s += g.w[i] * f(mid + 0.5 * h * g.x[i]);
    }
    return s * 0.5 * h;
}

// Panels of the 64-point rule for int_{a0}^{a1} of a function analytic away
// from a = 0: each panel no longer than the distance of the interval from 0,
// so that the rule's error (below rho^-128 with rho >= 2 + sqrt 3 for
// singularities at least a panel's length away) is far under FP64 rounding.
// A time step (a1 - a0 <= a0) takes one panel.
int panels_for(double a0, double a1) {
    const double lo = std::min(a0, a1), len = std::fabs(a1 - a0);
    if (!(lo > 0.0)) return 16;
    return (int)std::min(16.0, std::max(1.0, std::ceil(len / lo)));
}

struct Cosmo {
    double om, ol;
    // the last two growth values g(a) (a step's g(a_to) is the next step's g(a_from))
    mutable double memo_a[2] = {-1.0, -1.0}, memo_g[2] = {0.0, 0.0};
    mutable int memo_next = 0;
    bool eds() const { return om == 1.0 && ol == 0.0; }
    double E(double a) const { return std::sqrt(om / (a * a * a) + (1.0 - om - ol) / (a * a) + ol); }
    // int da / (a^2 E): kick factor
    double kick(double a0, double a1) const {
        if (a1 == a0) return 0.0;
        if (eds()) return 2.0 * (std::sqrt(a1) - std::sqrt(a0));
        return integrate([&](double a) { return 1.0 / (a * a * E(a)); }, a0, a1, panels_for(a0, a1));
    }
    // int da / (a^3 E): drift factor
    double drift(double a0, double a1) const {
        if (a1 == a0) return 0.0;
        if (eds()) return 2.0 * (1.0 / std::sqrt(a0) - 1.0 / std::sqrt(a1));
        return integrate([&](double a) { return 1.0 / (a * a * a * E(a)); }, a0, a1, panels_for(a0, a1));
    }
    // Heath integral int_0^a dx / (x E(x))^3, with x = t^2 to smooth the origin
    double heath(double a) const {
        return integrate([&](double t) {
            if (t == 0.0) return 0.0;
            double x = t * t, xe = x * E(x);
            return 2.0 * t / (xe * xe * xe);
        }, 0.0, std::sqrt(a));
    }
    // momentum growth g = a^2 E f D with D = (5/2) Om E heath (unnormalised:
    // the normalisation cancels in ratios) and f = d ln D / d ln a
    double g(double a) const {
        if (eds()) return a * std::sqrt(a);
        for (int i = 0; i < 2; ++i)
            if (memo_a[i] == a) return memo_g[i];
        const double h = heath(a), e = E(a), ok = 1.0 - om - ol;
        const double D = 2.5 * om * e * h;
        const double f = (-1.5 * om / (a * a * a) - ok / (a * a)) / (e * e) + 1.0 / (a * a * e * e * e * h);
        const double v = a * a * e * f * D;
        memo_a[memo_next] = a;
        memo_g[memo_next] = v;
        memo_next ^= 1;
        return v;
    }
};

// The largest a in (a0, hi] with h(a) <= limit, for h increasing with
// h(a0) <= limit < h(hi) and derivative dh: Newton's method on h = limit
// from the tangent at a0 (below the root when h is concave, as the drift
// integral is), kept inside the bracket (bisection where a step leaves it),
// then the root estimate stepped down by a few ulps until it meets the limit.
template <class H, class DH>
double largest_within(H h, DH dh, double a0, double hi, double limit) {
    double lo = a0, up = hi, x = hi;
    const double d0 = dh(a0);
    if (d0 > 0.0) {
        const double t = a0 + (limit - h(a0)) / d0;
        if (t > a0 && t < hi) x = t;
    }
    for (int it = 0; it < 100; ++it) {
        const double hx = h(x);
        if (hx <= limit) lo = std::max(lo, x);
        else up = std::min(up, x);
        const double d = dh(x);
        const double step = d > 0.0 ? (hx - limit) / d : 0.0;
        if (d > 0.0 && std::fabs(step) <= 1e-15 * x) break;       // x is the root to rounding
        if (up - lo <= 1e-15 * up) {
            x = lo;
            break;
        }
        double nx = d > 0.0 ? x - step : 0.5 * (lo + up);
        if (!(nx > lo && nx < up)) nx = 0.5 * (lo + up);
        x = nx;
    }
    for (int k = 0; k < 64 && x > lo; ++k) {
        if (h(x) <= limit) return x;
        x = std::max(lo, x - std::ldexp(x, -50) * (k + 1));
    }
    return lo;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool is_2a3b(int n) {
    if (n <= 0) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

double sinc(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }

}  // namespace

void cube::set_last_error(const std::string& msg) { g_err = msg; }

struct cube_ctx {
    cube_params P{};
    Geo g{};
    Cosmo cosmo{};
    cudaStream_t st = nullptr;
    int device = 0;
    // store, double-buffered: the step reads [cur] and writes [1 - cur]
    unsigned* counts[2] = {nullptr, nullptr};
    unsigned* offsets[2] = {nullptr, nullptr};
    float* vc[2] = {nullptr, nullptr};
    void* chi[2] = {nullptr, nullptr};
    void* nu[2] = {nullptr, nullptr};
    unsigned* id[2] = {nullptr, nullptr};
    int cur = 0;
    // velocity codec tables, [cur] describes the current store
    double* tanv = nullptr;
    double* tanh_ = nullptr;
    CodecDev codec[2]{};
    bool raw = false;               // uncompressed FP32 store: chi[0] = positions, nu[0] = momenta
    // per-step scratch
    long long* vsum = nullptr;
    unsigned* ghost = nullptr;
    float* part = nullptr;
    int npart = 0;
    unsigned* flags = nullptr;
    int* maxmig = nullptr;
    bool phig_valid = false;        // phig holds the potential of the last step or cube_potential call
    unsigned* scan_tmp = nullptr;
    long long* mom = nullptr;
    unsigned* vmax = nullptr;       // largest |p| of the store, float bits
    float* mesh = nullptr;
    float* phig = nullptr;          // ghosted Phi, written by the c2r sweep
    CUtensorMap phig_map{};         // TMA map of phig with pass A's tile as the box
    bool tma = false;               // phig_map encoded (else pass A loads with cp.async)
    FftPlan fft{};
    // host-pointer staging (lazily allocated when the work slab's region is too small)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    double stage_sigma = 0.0;           // host copy of a loaded codec scale (source of its upload)
    // device memory in two slabs: the state kept between calls (store, codec
    // tables, small results) and the work buffers of one call (mesh, ghosted
    // Phi, histograms, scan scratch, host staging).  A standalone context owns
    // both; a server's context owns its state slab (stream-ordered) and is
    // bound to its stream's shared work slab before each use.
    char* state_slab = nullptr;
    size_t state_size = 0;
    char* work_slab = nullptr;          // owned work slab (standalone contexts)
    size_t work_size = 0;
    char* work_base = nullptr;          // the work slab in use
    void* stage_ws = nullptr;           // host-staging region of the work slab
    size_t stage_ws_bytes = 0;
    bool served = false;
    bool member = false;                // a batch member: its slab belongs to the batch
    // drifted-state export
    bool keep = false;
    int* dbg_cell = nullptr;
    float* dbg_u = nullptr;
    float* dbg_p = nullptr;
    float* dbg_f = nullptr;
    bool dbg_valid = false;
    // host mirror of the state
    bool encoded = false;
    double a = 0.0, a_p = 0.0;
    int64_t steps = 0;
    uint64_t version = 0;           // changes whenever the store does (encode, step, checkpoint load)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    int64_t launches = 0;               // kernels launched by this context
    // per-kernel tracing: CUBE_PHASES + 1 boundary events per traced step
    int prof_max = 0, prof_steps = 0;
    std::vector<cudaEvent_t> prof_ev;

    StoreDev store(int k) const { return StoreDev{counts[k], offsets[k], vc[k], chi[k], nu[k], id[k]}; }
};

namespace {

// next 256-byte aligned piece of a slab (base == nullptr: sizing pass)
template <class T>
void carve(char* base, size_t& off, T*& p, size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes ? bytes : 16;
}

// device state of a context: both stores, codec tables and small results
size_t state_layout(cube_ctx* c, char* base) {
    const Geo& g = c->g;
    const size_t Np = (size_t)g.Np, Ncc = (size_t)g.Ncc;
    size_t off = 0;
    for (int k = 0; k < 2; ++k) {
        carve(base, off, c->counts[k], Ncc * 4);
        carve(base, off, c->offsets[k], (Ncc + 1) * 4);
        carve(base, off, c->vc[k], 3 * Ncc * 4);
        if (k == 0 || !c->raw) {         // the uncompressed store is updated in place
            carve(base, off, c->chi[k], 3 * Np * g.nchi);
            carve(base, off, c->nu[k], 3 * Np * g.nnu);
            if (c->P.id_bytes) carve(base, off, c->id[k], Np * (size_t)c->P.id_bytes);
        }
        carve(base, off, c->codec[k].dec, (size_t)(2 * g.nulim + 1) * 4);
        carve(base, off, c->codec[k].thr, (size_t)(g.nulim + 2) * 4);
        carve(base, off, c->codec[k].est, 8 * 4);
        carve(base, off, c->codec[k].vtab, VT_N);
        carve(base, off, c->codec[k].sigma, 8);
        if (g.nnu == 2) carve(base, off, c->codec[k].vdel, (size_t)g.nulim + 2);
    }
    carve(base, off, c->tanv, (size_t)(g.nulim + 1) * 8);
    carve(base, off, c->tanh_, (size_t)(g.nulim + 2) * 8);
    carve(base, off, c->flags, 4);
    carve(base, off, c->maxmig, ((size_t)g.nbricks + 2) * 4);    // [0] max migration, [1 ..] crowded-brick list
    carve(base, off, c->mom, 4 * 8);
    carve(base, off, c->vmax, 4);
    FftPlan& f = c->fft;
    carve(base, off, f.tw, (size_t)g.N * 8);
    carve(base, off, f.k2, (size_t)g.N * 4);
    carve(base, off, f.wdec, (size_t)g.N * 4);
    carve(base, off, f.wpk, (size_t)g.N * 8);
    return off;
}

// bytes of host staging and encode scratch: keys, permutation and radix
// workspace, then the particles when they come from host memory
size_t encode_scratch_bytes(const Geo& g, bool host) {
    const size_t Np = (size_t)g.Np;
    return (size_t)(2 * Np + radix_tmp_words(g.Np)) * 4 + (host ? 28 * Np : 0);
}

// work buffers of one call: mesh, ghosted Phi, step histograms and partial
// sums, scan scratch, and a staging region for host-array encode and decode
size_t work_layout(cube_ctx* c, char* base) {
    const Geo& g = c->g;
    const size_t Ncc = (size_t)g.Ncc;
    const int H3 = g.Bh * g.Bh * g.Bh;
    size_t off = 0;
    carve(base, off, c->mesh, (size_t)g.N * g.N * g.S * 4);
    carve(base, off, c->phig, (size_t)phig_nx(g.N) * phig_ny(g.N) * phig_ny(g.N) * 4);
    carve(base, off, c->vsum, 3 * Ncc * 8);
    carve(base, off, c->ghost, ((size_t)g.nbricks * H3 + 1) * 4);
    c->npart = std::max(g.nbricks, 1024);
    carve(base, off, c->part, (size_t)c->npart * 4);
    carve(base, off, c->scan_tmp,
          (size_t)scan_tmp_words(std::max<int64_t>(g.Ncc + 1, (int64_t)g.nbricks * H3 + 1)) * 4 + 64);
    c->stage_ws_bytes = c->raw ? 28 * (size_t)g.Np : encode_scratch_bytes(g, true);
    carve(base, off, c->stage_ws, c->stage_ws_bytes);
    return off;
}

cube_status stage_bytes(cube_ctx* c, size_t bytes, void** out) {
    if (c->stage_ws && bytes <= c->stage_ws_bytes) {   // the work slab's staging region
        *out = c->stage_ws;
        return CUBE_OK;
    }
    if (c->stage_bytes < bytes) {
        if (c->stage) cudaFree(c->stage);
        c->stage = nullptr;
        c->stage_bytes = 0;
        CK(cudaMalloc(&c->stage, bytes));
        c->stage_bytes = bytes;
    }
    *out = c->stage;
    return CUBE_OK;
}

cube_status flags_status(unsigned f) {
    if (f & ERR_MIGRATION) return fail(CUBE_E_MIGRATION, "a particle moved more than one coarse cell in a step");
    if (f & ERR_NONFINITE) return fail(CUBE_E_OVERFLOW, "non-finite particle position or velocity");
    if (f & ERR_COUNT) return fail(CUBE_E_OVERFLOW, "cell counts inconsistent with the particle total");
    if (f & ERR_TIMEOUT) return fail(CUBE_E_TIMEOUT, "a bounded wait for an asynchronous tile copy gave up");
    return CUBE_OK;
}

cube_status latched(cube_ctx* c) {
    unsigned f = 0;
    CK(cudaMemcpyAsync(&f, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return flags_status(f);
}

// TMA descriptor of the ghosted Phi: a 3-D float tensor (x, y, z extents
// N + 8, N + 5, N + 5) whose box is pass A's tile ((F + 8) x (F + 5) x (F + 5)).
// The encoder comes from the driver through the runtime; any failure leaves
// pass A on its cp.async path.
bool encode_phig_map(const Geo& g, float* phig, int members, size_t stride, CUtensorMap* out) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&enc, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !enc) {
        cudaGetLastError();
        return false;
    }
    const cuuint64_t plane = (cuuint64_t)phig_nx(g.N) * phig_ny(g.N) * 4;
    // 4-D: x, y, z and the member of a batch (one member: any stride that is a multiple of 16)
    const cuuint64_t dims[4] = {(cuuint64_t)phig_nx(g.N), (cuuint64_t)phig_ny(g.N), (cuuint64_t)phig_ny(g.N),
                                (cuuint64_t)members};
    const cuuint64_t strides[3] = {(cuuint64_t)phig_nx(g.N) * 4, plane,
                                   members > 1 ? (cuuint64_t)stride : plane * phig_ny(g.N)};
    const cuuint32_t box[4] = {(cuuint32_t)(g.F + 8), (cuuint32_t)(g.F + 5), (cuuint32_t)(g.F + 5), 1};
    const cuuint32_t unit[4] = {1, 1, 1, 1};
    const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, phig, dims, strides, box, unit,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_phig_map(cube_ctx* c) { return encode_phig_map(c->g, c->phig, 1, 0, &c->phig_map); }

// geometry and flags of a context from validated parameters (brick side B)
void init_geo(cube_ctx* c, const cube_params* params, int B) {
    c->P = *params;
    c->cosmo = Cosmo{params->omega_m, params->omega_l};
    Geo& g = c->g;
    g.N = params->n_fine;
    g.R = params->ratio;
    g.r = g.R == 1 ? 0 : g.R == 2 ? 1 : g.R == 4 ? 2 : 3;
    g.Nc = g.N / g.R;
    g.B = B;
    g.nb = g.Nc / B;
    g.Bh = B + 2;
    c->raw = params->x_bytes == 4;
    g.nchi = c->raw ? 4 : params->x_bytes;
    g.nnu = c->raw ? 4 : params->v_bytes;
    g.sbits = 8 * g.nchi + 1 - g.r;
    g.F = B * g.R;
    g.S = g.N + 4;
    g.Ncc = g.Nc * g.Nc * g.Nc;
    g.nbricks = g.nb * g.nb * g.nb;
    g.Np = params->n_particles;
    g.nulim = c->raw ? 127 : (1 << (8 * g.nnu - 1)) - 1;   // (no codec tables are used uncompressed)
    g.nid = params->id_bytes;
    g.lB = 0;
    while ((1 << g.lB) < g.B) ++g.lB;
    g.lF = 0;
    while ((1 << g.lF) < g.F) ++g.lF;
    g.nsm = 1;
    c->fft.N = g.N;
}

cube_status check_params(const cube_params* p, int* brick) {
    if (!p) return fail(CUBE_E_ARG, "params is NULL");
    const int N = p->n_fine;
    if (N < 16 || N > 1024 || !is_2a3b(N) || !fft_size_supported(N))
        return fail(CUBE_E_ARG, "n_fine must be 2^a or 3 * 2^a in [16, 1024]");
    const int R = p->ratio;
    if (!(R == 1 || R == 2 || R == 4 || R == 8) || N % R) return fail(CUBE_E_ARG, "ratio must be 1, 2, 4 or 8 and divide n_fine");
    const int Nc = N / R;
    if (Nc < 3) return fail(CUBE_E_ARG, "need at least 3 coarse cells per side");
    if (p->n_particles < 1 || p->n_particles >= (1LL << 31)) return fail(CUBE_E_ARG, "n_particles out of range");
    const bool raw = p->x_bytes == 4 && p->v_bytes == 4;
    if (!raw && ((p->x_bytes != 1 && p->x_bytes != 2) || (p->v_bytes != 1 && p->v_bytes != 2)))
        return fail(CUBE_E_ARG, "x_bytes and v_bytes must be 1 or 2 (codes), or both 4 (uncompressed FP32)");
    if (p->id_bytes != 0 && p->id_bytes != 1 && p->id_bytes != 2 && p->id_bytes != 4)
        return fail(CUBE_E_ARG, "id_bytes must be 0, 1, 2 or 4");
    if (raw && p->id_bytes != 0 && p->id_bytes != 4)
        return fail(CUBE_E_ARG, "the uncompressed store keeps 4-byte particle IDs (id_bytes 0 or 4)");
    if (p->gradient != CUBE_GRAD_FD4) return fail(CUBE_E_ARG, "only CUBE_GRAD_FD4 is implemented");
    if (p->deconv_power < 0 || p->deconv_power > 2) return fail(CUBE_E_ARG, "deconv_power must be 0, 1 or 2");
    if (!(p->box > 0.0) || !(p->omega_m > 0.0) || !(p->omega_l >= 0.0)) return fail(CUBE_E_ARG, "box, omega_m must be > 0");
    int B = p->brick;
    if (B == 0) {
        const int cand[3] = {4, 2, 1};
        for (int b : cand)
            if (Nc % b == 0 && Nc / b >= 3 && b * R <= 16 && b * R >= 4) { B = b; break; }
        if (B == 0) return fail(CUBE_E_ARG, "no valid brick size");
    }
    if (!(B == 1 || B == 2 || B == 4) || Nc % B || Nc / B < 3 || B * R > 16 || B * R < 4)
        return fail(CUBE_E_ARG, "brick must be 1, 2 or 4, divide N_c with >= 3 bricks per side, "
                                "and 4 <= brick * ratio <= 16");
    *brick = B;
    return CUBE_OK;
}

}  // namespace

extern "C" {

const char* cube_last_error(void) { return g_err.c_str(); }

cube_status cube_destroy(cube_ctx* c) {
    if (!c) return CUBE_OK;
    if (c->member) {                     // the batch frees the slab
        cudaStreamSynchronize(c->st);
    } else if (c->served) {              // stream-ordered: no device-wide synchronisation
        if (c->state_slab) cudaFreeAsync(c->state_slab, c->st);
    } else {
        cudaStreamSynchronize(c->st);
        if (c->state_slab) cudaFree(c->state_slab);
        if (c->work_slab) cudaFree(c->work_slab);
    }
    if (c->stage) cudaFree(c->stage);
    if (c->dbg_cell) cudaFree(c->dbg_cell);
    if (c->dbg_u) cudaFree(c->dbg_u);
    if (c->dbg_p) cudaFree(c->dbg_p);
    if (c->dbg_f) cudaFree(c->dbg_f);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
    return CUBE_OK;
}

// member_base: a batch member's device slab (state, then work at the next
// 256-byte boundary), allocated by the batch; null: the context allocates
static cube_status create_ctx(const cube_params* params, void* cuda_stream, bool served, cube_ctx** out,
                              char* member_base = nullptr) {
    if (!out) return fail(CUBE_E_ARG, "out is NULL");
    *out = nullptr;
    int B = 0;
    cube_status s = check_params(params, &B);
    if (s != CUBE_OK) return s;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    cube_ctx* c = new cube_ctx();
    c->st = (cudaStream_t)cuda_stream;
    c->served = served;
    cudaGetDevice(&c->device);
    init_geo(c, params, B);
    const Geo& g = c->g;
    cudaDeviceGetAttribute(&c->g.nsm, cudaDevAttrMultiProcessorCount, c->device);

    auto bad = [&](cudaError_t e, const char* what) -> cube_status {
        cube_destroy(c);
        return fail(e == cudaErrorMemoryAllocation ? CUBE_E_NOMEM : CUBE_E_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    };
    c->state_size = state_layout(c, nullptr);
    c->work_size = work_layout(c, nullptr);
    if (member_base) {
        c->member = true;
        state_layout(c, member_base);
        c->work_base = member_base + ((c->state_size + 255) & ~(size_t)255);
        work_layout(c, c->work_base);
    } else {
        {
            cudaError_t e = c->served ? cudaMallocAsync((void**)&c->state_slab, c->state_size, c->st)
                                      : cudaMalloc((void**)&c->state_slab, c->state_size);
            if (e == cudaSuccess && !c->served) e = cudaMalloc((void**)&c->work_slab, c->work_size);
            if (e != cudaSuccess) return bad(e, "device memory");
        }
        state_layout(c, c->state_slab);
        if (!c->served) {
            c->work_base = c->work_slab;
            work_layout(c, c->work_base);
        }
    }
    FftPlan& f = c->fft;
    // host tables (FP64 libm), uploaded once (stream-ordered: pageable sources are
    // staged before each call returns)
    {
        std::vector<float2> tw(g.N);
        std::vector<float> k2(g.N), wd(g.N);
        std::vector<double> wpk(g.N);
        for (int i = 0; i < g.N; ++i) {
            double ang = 2.0 * PI * i / g.N;
            tw[i] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
            int fr = i <= g.N / 2 ? i : i - g.N;
            double kk = 2.0 * PI * fr / g.N;
            k2[i] = (float)(kk * kk);
            double sn = sinc(PI * fr / g.N);
            wd[i] = (float)std::pow(sn, -2.0 * params->deconv_power);
            wpk[i] = std::pow(sn, -4.0);
        }
        const int M = 2 * g.nulim + 1;
        std::vector<double> tv(g.nulim + 1), th(g.nulim + 2);
        for (int k = 0; k <= g.nulim; ++k) tv[k] = std::tan(PI * k / M);
        for (int k = 0; k <= g.nulim + 1; ++k) th[k] = std::tan(PI * (k - 0.5) / M);
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaMemcpyAsync(f.tw, tw.data(), g.N * 8, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f.k2, k2.data(), g.N * 4, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f.wdec, wd.data(), g.N * 4, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f.wpk, wpk.data(), g.N * 8, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->tanv, tv.data(), tv.size() * 8, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->tanh_, th.data(), th.size() * 8, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, 4, c->st);
        if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
        if (e != cudaSuccess) return bad(e, "table upload");
    }
    c->tma = c->phig ? encode_phig_map(c) : false;     // a server's context: at its first binding
    *out = c;
    return CUBE_OK;
}

cube_status cube_create(const cube_params* params, void* cuda_stream, cube_ctx** out) {
    return create_ctx(params, cuda_stream, false, out);
}

// Uncompressed store: copy (and wrap) the particles; momenta and positions share the epoch a.
static cube_status raw_encode(cube_ctx* c, const float* pos, const float* vel, const uint32_t* id, double a,
                              bool hpos, bool hvel, bool hid, bool sync) {
    const Geo& g = c->g;
    const size_t Np = (size_t)g.Np;
    const size_t need = (hpos ? 12 * Np : 0) + (hvel ? 12 * Np : 0) + (hid ? 4 * Np : 0);
    char* sp = nullptr;
    if (need) {
        void* p = nullptr;
        cube_status s = stage_bytes(c, need, &p);
        if (s != CUBE_OK) return s;
        sp = (char*)p;
    }
    const float* dpos = pos;
    const float* dvel = vel;
    const unsigned* did = id;
    if (hpos) { CK(cudaMemcpyAsync(sp, pos, 12 * Np, cudaMemcpyHostToDevice, c->st)); dpos = (const float*)sp; sp += 12 * Np; }
    if (hvel) { CK(cudaMemcpyAsync(sp, vel, 12 * Np, cudaMemcpyHostToDevice, c->st)); dvel = (const float*)sp; sp += 12 * Np; }
    if (hid) { CK(cudaMemcpyAsync(sp, id, 4 * Np, cudaMemcpyHostToDevice, c->st)); did = (const unsigned*)sp; }
    CK(cudaMemsetAsync(c->flags, 0, 4, c->st));
    CK(cudaMemsetAsync(c->maxmig, 0, 4, c->st));
    launch_raw_encode(g, dpos, dvel, did, (float*)c->chi[0], (float*)c->nu[0], c->id[0], c->flags, c->st);
    c->launches += 1;
    CK(cudaGetLastError());
    if (sync) CK(cudaStreamSynchronize(c->st));
    c->cur = 0;
    c->encoded = true;
    c->phig_valid = false;
    c->a = a;
    c->a_p = a;
    c->steps = 0;
    c->version += 1;
    c->dbg_valid = false;
    c->timed = false;
    return CUBE_OK;
}

// encode, enqueued on the context's stream; sync: wait for it (host arrays
// may then be released and the staging reused at once)
static cube_status encode_impl(cube_ctx* c, const float* pos, const float* vel, const uint32_t* id, double a,
                               double sigma, bool sync) {
    if (!c) return fail(CUBE_E_ARG, "ctx is NULL");
    if (!pos || !vel) return fail(CUBE_E_ARG, "pos and vel are required");
    if (!(a > 0.0)) return fail(CUBE_E_ARG, "a must be > 0");
    const Geo& g = c->g;
    const size_t Np = (size_t)g.Np;
    const bool hpos = !is_device_ptr(pos), hvel = !is_device_ptr(vel), hid = id && !is_device_ptr(id);
    if (c->raw) return raw_encode(c, pos, vel, id, a, hpos, hvel, hid, sync);
    // scratch: keys, perm, radix workspace, host staging
    const int key_bits = std::max(1, (int)std::ceil(std::log2((double)g.Ncc)));
    size_t words = (size_t)(2 * Np) + (size_t)radix_tmp_words(g.Np);
    size_t stage_off = words * 4;
    size_t need = stage_off + (hpos ? 12 * Np : 0) + (hvel ? 12 * Np : 0) + (hid ? 4 * Np : 0);
    void* scratch = nullptr;
    cube_status s = stage_bytes(c, need, &scratch);
    if (s != CUBE_OK) return s;
    unsigned* keys = (unsigned*)scratch;
    unsigned* perm = keys + Np;
    unsigned* rtmp = perm + Np;
    char* sp = (char*)scratch + stage_off;
    const float* dpos = pos;
    const float* dvel = vel;
    const unsigned* did = id;
    if (hpos) { CK(cudaMemcpyAsync(sp, pos, 12 * Np, cudaMemcpyHostToDevice, c->st)); dpos = (const float*)sp; sp += 12 * Np; }
    if (hvel) { CK(cudaMemcpyAsync(sp, vel, 12 * Np, cudaMemcpyHostToDevice, c->st)); dvel = (const float*)sp; sp += 12 * Np; }
    if (hid) { CK(cudaMemcpyAsync(sp, id, 4 * Np, cudaMemcpyHostToDevice, c->st)); did = (const unsigned*)sp; }
    c->cur = 0;                          // a fresh store always starts in buffer 0 (batch members stay in step)
    const int k = c->cur;
    CK(cudaMemsetAsync(c->flags, 0, 4, c->st));
    CK(cudaMemsetAsync(c->counts[k], 0, (size_t)g.Ncc * 4, c->st));
    CK(cudaMemsetAsync(c->vsum, 0, (size_t)g.Ncc * 24, c->st));
    launch_encode_keys(g, dpos, dvel, keys, perm, c->counts[k], c->vsum, c->flags, c->st);
    exclusive_scan(c->counts[k], c->offsets[k], g.Ncc, c->scan_tmp, c->st);
    launch_vc_finalize(g, c->counts[k], c->vsum, c->vc[k], c->st);
    if (sigma > 0.0) {
        launch_sigma_finalize(c->part, 0, 1.0, 1.0, sigma, c->codec[k].sigma, c->st);
    } else {
        launch_encode_sigma(g, dvel, keys, c->vc[k], c->part, c->st);
        launch_sigma_finalize(c->part, encode_sigma_blocks(g), 3.0 * (double)g.Np, 1.0, 0.0, c->codec[k].sigma, c->st);
    }
    launch_codec_tables(g.nulim, c->tanv, c->tanh_, c->codec[k], c->st);
    radix_sort_pairs(keys, perm, g.Np, key_bits, rtmp, c->st);
    launch_encode_scatter(g, dpos, dvel, did, keys, perm, c->vc[k], c->codec[k], c->store(k), c->st);
    c->launches += 1 + 4 + 1 + (sigma > 0.0 ? 1 : 2) + 1 + (int64_t)((key_bits + 7) / 8) * 6 + 1;
    CK(cudaGetLastError());
    if (sync) CK(cudaStreamSynchronize(c->st));
    c->encoded = true;
    c->phig_valid = false;
    c->a = a;
    c->a_p = a;
    c->steps = 0;
    c->version += 1;
    c->dbg_valid = false;
    c->timed = false;
    return CUBE_OK;
}

cube_status cube_encode(cube_ctx* c, const float* pos, const float* vel, const uint32_t* id, double a, double sigma) {
    return encode_impl(c, pos, vel, id, a, sigma, true);
}

// kernels launched per phase of a step (see cube_phase_name)
const int kPhaseKernels[CUBE_PHASES] = {0, 1, 1, 1, 1, 1, 1, 1, 2, 4, 1, 1};
const char* kPhaseNames[CUBE_PHASES] = {"setup", "deposit", "fft_x_r2c", "fft_y_fwd", "fft_z_green", "fft_y_inv",
                                        "fft_x_c2r", "pass_a", "codec", "scan", "cells", "pass_b"};

// the uncompressed store's step: mesh cleared in setup, one deposit, the FFT
// sweeps, one kick-drift kernel in the pass_a slot
const int kPhaseKernelsRaw[CUBE_PHASES] = {0, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0};

static void mark(cube_ctx* c, int boundary) {
    if (c->prof_steps < c->prof_max) cudaEventRecord(c->prof_ev[(size_t)c->prof_steps * (CUBE_PHASES + 1) + boundary], c->st);
}

static double particle_mass(const Geo& g) { return std::pow((double)g.N, 3) / (double)g.Np; }

static void deposit(cube_ctx* c) {
    const Geo& g = c->g;
    if (c->raw) {
        cudaMemsetAsync(c->mesh, 0, (size_t)g.N * g.N * g.S * 4, c->st);
        launch_raw_deposit(g, (const float*)c->chi[0], c->mesh, (float)particle_mass(g), c->st);
    } else {
        launch_deposit(g, c->store(c->cur), c->mesh, particle_mass(g) * std::ldexp(1.0, -3 * g.sbits), c->st);
    }
    c->launches += 1;
}

// density -> Phi on the mesh; boundaries 1..6 of the step's trace
static void mesh_potential(cube_ctx* c) {
    const Geo& g = c->g;
    deposit(c);
    mark(c, 2);
    fft_x_r2c(c->fft, c->mesh, g.S, c->st);
    mark(c, 3);
    fft_y(c->fft, c->mesh, g.S, false, c->st);
    mark(c, 4);
    const float g0 = (float)(-1.5 * c->P.omega_m / std::pow((double)g.N, 3));
    fft_z(c->fft, c->mesh, g.S, g0, true, c->st);
    mark(c, 5);
    fft_y(c->fft, c->mesh, g.S, true, c->st);
    mark(c, 6);
    fft_x_c2r(c->fft, c->mesh, g.S, c->phig, c->st);
    mark(c, 7);
    c->launches += 5;
}

cube_status cube_pm_step(cube_ctx* c, double a_from, double a_to) {
    if (!c) return fail(CUBE_E_ARG, "ctx is NULL");
    if (!c->encoded) return fail(CUBE_E_STATE, "cube_pm_step before cube_encode");
    if (std::fabs(a_from - c->a) > 1e-12 * std::max(1.0, std::fabs(a_from)))
        return fail(CUBE_E_STATE, "a_from differs from the store's epoch");
    if (!(a_to > a_from)) return fail(CUBE_E_ARG, "a_to must exceed a_from");
    const Geo& g = c->g;
    const double a_mid = 0.5 * (a_from + a_to);
    const float kick = (float)c->cosmo.kick(c->a_p, a_mid);
    const float dc = (float)(c->cosmo.drift(a_from, a_to) / g.R);
    const double ratio = c->cosmo.g(a_to) / c->cosmo.g(a_from);
    if (c->raw) {
        CK(cudaEventRecord(c->ev0, c->st));
        mark(c, 0);
        mark(c, 1);
        mesh_potential(c);
        c->phig_valid = true;
        launch_raw_kick_drift(g, (float*)c->chi[0], (float*)c->nu[0], c->phig, kick,
                              (float)c->cosmo.drift(a_from, a_to), c->flags, c->st);
        for (int b = 8; b <= 12; ++b) mark(c, b);
        CK(cudaEventRecord(c->ev1, c->st));
        c->launches += 1;
        if (c->prof_steps < c->prof_max) c->prof_steps += 1;
        CK(cudaGetLastError());
        c->a = a_to;
        c->a_p = a_mid;
        c->steps += 1;
        c->version += 1;
        c->timed = true;
        return CUBE_OK;
    }
    const int k = c->cur, kn = 1 - k;
    if (c->keep) {
        if (!c->dbg_cell) {
            CK(cudaMalloc((void**)&c->dbg_cell, 12 * (size_t)g.Np));
            CK(cudaMalloc((void**)&c->dbg_u, 12 * (size_t)g.Np));
            CK(cudaMalloc((void**)&c->dbg_p, 12 * (size_t)g.Np));
            CK(cudaMalloc((void**)&c->dbg_f, 12 * (size_t)g.Np));
        }
    }
    CK(cudaEventRecord(c->ev0, c->st));
    mark(c, 0);
    CK(cudaMemsetAsync(c->vsum, 0, (size_t)g.Ncc * 24, c->st));
    CK(cudaMemsetAsync(c->maxmig, 0, 8, c->st));     // max migration, crowded-brick count
    mark(c, 1);
    mesh_potential(c);
    c->phig_valid = true;
    StepScratch w{c->counts[kn], c->vsum, c->ghost, c->part, c->flags, c->maxmig, c->maxmig + 1};
    DriftDebug dbg{c->keep ? c->dbg_cell : nullptr, c->dbg_u, c->dbg_p, c->dbg_f};
    launch_passA(g, c->store(k), c->phig, c->tma ? &c->phig_map : nullptr, c->codec[k], kick, dc, w, dbg, c->st);
    mark(c, 8);
    launch_sigma_finalize(c->part, g.nbricks, 3.0 * (double)g.Np, ratio, 0.0, c->codec[kn].sigma, c->st);
    launch_codec_tables(g.nulim, c->tanv, c->tanh_, c->codec[kn], c->st);
    mark(c, 9);
    exclusive_scan(c->ghost, c->ghost, (int64_t)g.nbricks * (g.Bh * g.Bh * g.Bh), c->scan_tmp, c->st);
    mark(c, 10);
    launch_cells(g, w, c->offsets[kn], c->vc[kn], c->st);
    mark(c, 11);
    launch_passB(g, c->store(k), c->store(kn), c->codec[k], c->codec[kn], dc, w, c->st);
    mark(c, 12);
    CK(cudaEventRecord(c->ev1, c->st));
    c->launches += 1 + 2 + 4 + 1 + 1;
    if (c->prof_steps < c->prof_max) c->prof_steps += 1;
    CK(cudaGetLastError());
    c->cur = kn;
    c->a = a_to;
    c->a_p = a_mid;
    c->steps += 1;
    c->version += 1;
    c->dbg_valid = c->keep;
    c->timed = true;
    return CUBE_OK;
}

static cube_status to_user(cube_ctx* c, void* dst, const void* src, size_t bytes, bool host) {
    CK(cudaMemcpyAsync(dst, src, bytes, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
    return CUBE_OK;
}

cube_status cube_decode(cube_ctx* c, float* pos, float* vel, uint32_t* id) {
    if (!c) return fail(CUBE_E_ARG, "ctx is NULL");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    if (!pos || !vel) return fail(CUBE_E_ARG, "pos and vel are required");
    const Geo& g = c->g;
    const size_t Np = (size_t)g.Np;
    const bool hpos = !is_device_ptr(pos), hvel = !is_device_ptr(vel), hid = id && !is_device_ptr(id);
    size_t need = (hpos ? 12 * Np : 0) + (hvel ? 12 * Np : 0) + (hid ? 4 * Np : 0);
    char* sp = nullptr;
    if (need) {
        void* p = nullptr;
        cube_status s = stage_bytes(c, need, &p);
        if (s != CUBE_OK) return s;
        sp = (char*)p;
    }
    float* dpos = hpos ? (float*)sp : pos;
    float* dvel = hvel ? (float*)(sp + (hpos ? 12 * Np : 0)) : vel;
    unsigned* did = id ? (hid ? (unsigned*)(sp + (hpos ? 12 * Np : 0) + (hvel ? 12 * Np : 0)) : id) : nullptr;
    if (c->raw) {                        // the store is the particles: copy them out
        CK(cudaMemcpyAsync(dpos, c->chi[0], 12 * Np, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(dvel, c->nu[0], 12 * Np, cudaMemcpyDeviceToDevice, c->st));
        if (did) {
            if (c->id[0]) CK(cudaMemcpyAsync(did, c->id[0], 4 * Np, cudaMemcpyDeviceToDevice, c->st));
            else launch_iota(did, g.Np, c->st);
        }
    } else {
        launch_decode(g, c->store(c->cur), c->codec[c->cur].dec, dpos, dvel, did, c->st);
        c->launches += 1;
    }
    CK(cudaGetLastError());
    cube_status s;
    if (hpos && (s = to_user(c, pos, dpos, 12 * Np, true)) != CUBE_OK) return s;
    if (hvel && (s = to_user(c, vel, dvel, 12 * Np, true)) != CUBE_OK) return s;
    if (hid && (s = to_user(c, id, did, 4 * Np, true)) != CUBE_OK) return s;
    return latched(c);
}

// P(k) of the current store, enqueued; k, pk, nmodes copied out (host copies
// are asynchronous only into pinned memory)
static cube_status pk_enqueue(cube_ctx* c, int32_t n_bins, double* k, double* pk, double* nmodes) {
    if (!c) return fail(CUBE_E_ARG, "ctx is NULL");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    if (n_bins < 1 || n_bins > 2048 || !k || !pk || !nmodes) return fail(CUBE_E_ARG, "n_bins in [1, 2048] and outputs required");
    const Geo& g = c->g;
    deposit(c);
    fft_x_r2c(c->fft, c->mesh, g.S, c->st);
    fft_y(c->fft, c->mesh, g.S, false, c->st);
    fft_z(c->fft, c->mesh, g.S, 0.0f, false, c->st);
    c->launches += 5;
    const int nb = pk_blocks(g.N);
    double* part = nullptr;
    double* outk = nullptr;
    size_t pbytes = (size_t)nb * 3 * n_bins * 8;
    CK(cudaMallocAsync((void**)&part, pbytes + 3 * (size_t)n_bins * 8, c->st));
    outk = part + (size_t)nb * 3 * n_bins;
    const double L = c->P.box;
    const double pfac = L * L * L / std::pow((double)g.N, 6);
    launch_pk_bin(c->fft, c->mesh, g.S, n_bins, pfac, 2.0 * PI / L, part, c->st);
    launch_pk_reduce(part, nb, n_bins, outk, outk + n_bins, outk + 2 * n_bins, c->st);
    c->launches += 2;
    cube_status s = CUBE_OK;
    const bool hk = !is_device_ptr(k), hp = !is_device_ptr(pk), hn = !is_device_ptr(nmodes);
    if ((s = to_user(c, k, outk, n_bins * 8, hk)) == CUBE_OK && (s = to_user(c, pk, outk + n_bins, n_bins * 8, hp)) == CUBE_OK)
        s = to_user(c, nmodes, outk + 2 * n_bins, n_bins * 8, hn);
    cudaFreeAsync(part, c->st);
    CK(cudaGetLastError());
    return s;
}

cube_status cube_power_spectrum(cube_ctx* c, int32_t n_bins, double* k, double* pk, double* nmodes) {
    cube_status s = pk_enqueue(c, n_bins, k, pk, nmodes);
    if (s != CUBE_OK) return s;
    return latched(c);
}

cube_status cube_max_speed(cube_ctx* c, double* p_max) {
    if (!c || !p_max) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    const Geo& g = c->g;
    if (c->raw) launch_raw_max_speed(g, (const float*)c->nu[0], c->vmax, c->st);
    else launch_max_speed(g, c->store(c->cur), c->codec[c->cur].dec, c->vmax, c->st);
    c->launches += 1;
    unsigned bits = 0;
    CK(cudaMemcpyAsync(&bits, c->vmax, 4, cudaMemcpyDeviceToHost, c->st));
    cube_status s = latched(c);
    float f;
    std::memcpy(&f, &bits, 4);
    *p_max = f;
    return s;
}

// largest a_to <= a_max with p * int_a^a_to da / (a^3 E) <= cells coarse cells
// (a = the store's epoch; drift(a, .) grows: bisection); a when none is
static double epoch_limit(const cube_ctx* c, double p, double a_max, double cells) {
    const double limit = cells * c->g.R;                 // fine cells
    const double a0 = c->a;
    const Cosmo& cm = c->cosmo;
    if (p * cm.drift(a0, a_max) <= limit) return a_max;
    return largest_within([&](double a) { return p * cm.drift(a0, a); },
                          [&](double a) { return p / (a * a * a * cm.E(a)); }, a0, a_max, limit);
}

cube_status cube_max_force(cube_ctx* c, double* f_max) {
    if (!c || !f_max) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    *f_max = 0.0;
    if (!c->phig_valid) return CUBE_OK;
    launch_grad_max(c->phig, c->g.N, c->vmax, c->st);
    c->launches += 1;
    unsigned bits = 0;
    CK(cudaMemcpyAsync(&bits, c->vmax, 4, cudaMemcpyDeviceToHost, c->st));
    cube_status s = latched(c);
    float f;
    std::memcpy(&f, &bits, 4);
    *f_max = f;
    return s;
}

static cube_status check_limits(const cube_step_limits* lim) {
    if (!(lim->drift_cells > 0.0 && lim->drift_cells <= 1.0)) return fail(CUBE_E_ARG, "drift_cells must be in (0, 1]");
    if (!(lim->max_dlna >= 0.0)) return fail(CUBE_E_ARG, "max_dlna must be >= 0");
    return CUBE_OK;
}

// Largest a_to <= a_max within the limits for positions at a0, momenta at
// a_p, fastest momentum p and largest force component f; R fine cells per
// coarse cell.  `why`: 0 a_max, 1 the drift, 2 the expansion limit.
static cube_status limited_epoch(const Cosmo& cosmo, int R, double a0, double a_p, double a_max, double p, double f,
                                 const cube_step_limits* lim, double* a_to, int32_t* binding) {
    const double limit = lim->drift_cells * R;
    // expansion: Delta ln a <= max_dlna
    double hi = a_max;
    int why = 0;
    if (lim->max_dlna > 0.0 && a0 * std::exp(lim->max_dlna) < hi) {
        hi = a0 * std::exp(lim->max_dlna);
        why = 2;
    }
    // drift of the fastest particle after the kick of the largest force, per axis:
    // (p_max + F_max int_{a_p}^{a_mid} da / (a^2 E)) int_a^{a_to} da / (a^3 E), increasing in a_to
    auto drift = [&](double at) { return (p + f * cosmo.kick(a_p, 0.5 * (a0 + at))) * cosmo.drift(a0, at); };
    if (drift(hi) <= limit) {
        *a_to = hi;
    } else {
        // d/da_to of the drift: the kick's growth times the drift factor, plus
        // the kicked momentum times the drift integrand
        auto slope = [&](double at) {
            const double am = 0.5 * (a0 + at);
            return 0.5 * f / (am * am * cosmo.E(am)) * cosmo.drift(a0, at) +
                   (p + f * cosmo.kick(a_p, am)) / (at * at * at * cosmo.E(at));
        };
        *a_to = largest_within(drift, slope, a0, hi, limit);
        why = 1;
    }
    if (binding) *binding = why;
    return *a_to > a0 ? CUBE_OK : fail(CUBE_E_ARG, "no step keeps the fastest particle within the limit");
}

cube_status cube_next_epoch_limited(cube_ctx* c, double a_max, const cube_step_limits* lim, double* a_to,
                                    int32_t* binding) {
    if (!c || !a_to || !lim) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    if (!(a_max > c->a)) return fail(CUBE_E_ARG, "a_max must exceed the store's epoch");
    cube_status s = check_limits(lim);
    if (s != CUBE_OK) return s;
    double p = 0.0, f = 0.0;
    s = cube_max_speed(c, &p);
    if (s == CUBE_OK) s = cube_max_force(c, &f);
    if (s != CUBE_OK) return s;
    return limited_epoch(c->cosmo, c->g.R, c->a, c->a_p, a_max, p, f, lim, a_to, binding);
}

cube_status cube_epoch_bound(double omega_m, double omega_l, int32_t ratio, double a, double a_p, double a_max,
                             double p_max, double f_max, const cube_step_limits* lim, double* a_to,
                             int32_t* binding) {
    if (!a_to || !lim) return fail(CUBE_E_ARG, "NULL argument");
    if (!(omega_m > 0.0) || !(omega_l >= 0.0)) return fail(CUBE_E_ARG, "omega_m must be > 0, omega_l >= 0");
    if (ratio < 1) return fail(CUBE_E_ARG, "ratio must be >= 1");
    if (!(a > 0.0) || !(a_p > 0.0) || !(a_p <= a)) return fail(CUBE_E_ARG, "need 0 < a_p <= a");
    if (!(a_max > a)) return fail(CUBE_E_ARG, "a_max must exceed a");
    if (!(p_max >= 0.0) || !(f_max >= 0.0)) return fail(CUBE_E_ARG, "p_max and f_max must be >= 0");
    cube_status s = check_limits(lim);
    if (s != CUBE_OK) return s;
    return limited_epoch(Cosmo{omega_m, omega_l}, ratio, a, a_p, a_max, p_max, f_max, lim, a_to, binding);
}

cube_status cube_leapfrog_factors(double omega_m, double omega_l, double a0, double a1, double* kick,
                                  double* drift, double* growth_ratio) {
    if (!(omega_m > 0.0) || !(omega_l >= 0.0)) return fail(CUBE_E_ARG, "omega_m must be > 0, omega_l >= 0");
    if (!(a0 > 0.0) || !(a1 > 0.0)) return fail(CUBE_E_ARG, "scale factors must be > 0");
    const Cosmo cosmo{omega_m, omega_l};
    if (kick) *kick = cosmo.kick(a0, a1);
    if (drift) *drift = cosmo.drift(a0, a1);
    if (growth_ratio) *growth_ratio = cosmo.g(a1) / cosmo.g(a0);
    return CUBE_OK;
}

cube_status cube_next_epoch(cube_ctx* c, double a_max, double cells, double* a_to) {
    if (!c || !a_to) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    if (!(a_max > c->a)) return fail(CUBE_E_ARG, "a_max must exceed the store's epoch");
    if (!(cells > 0.0 && cells <= 1.0)) return fail(CUBE_E_ARG, "cells must be in (0, 1]");
    double p = 0.0;
    cube_status s = cube_max_speed(c, &p);
    if (s != CUBE_OK) return s;
    *a_to = epoch_limit(c, p, a_max, cells);
    return *a_to > c->a ? CUBE_OK : fail(CUBE_E_ARG, "no step keeps the fastest particle within the limit");
}

// ---------------------------------------------------------------- checkpoint (Section 2.3.1)
// Layout: a 64-byte header, then 16-byte aligned sections.  Compressed store:
// counts u32[Ncc] (rho_c), v_c f32[3][Ncc], chi [3][N] codes, nu [3][N]
// codes, ids u32[N] (id_bytes 4).  Uncompressed store: positions f32[3][N],
// momenta f32[3][N], ids.
namespace {

struct CkptHeader {
    char magic[8];                       // "CUBECKP1"
    int32_t n_fine, ratio;
    int64_t n_particles;
    int32_t x_bytes, v_bytes, id_bytes, brick;
    double a, a_p, sigma;
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// byte offsets of the sections (sec[0..4]) and the total
size_t ckpt_layout(const Geo& g, bool raw, int id_bytes, size_t sec[5]) {
    const size_t N = (size_t)g.Np, Ncc = (size_t)g.Ncc;
    size_t off = sizeof(CkptHeader);
    const size_t sz[5] = {raw ? 12 * N : 4 * Ncc, raw ? 12 * N : 12 * Ncc, raw ? 0 : 3 * N * g.nchi,
                          raw ? 0 : 3 * N * g.nnu, (size_t)id_bytes * N};
    for (int i = 0; i < 5; ++i) {
        sec[i] = off;
        off = align16(off + sz[i]);
    }
    return off;
}

}  // namespace

cube_status cube_checkpoint_size(const cube_params* params, int64_t* bytes) {
    if (!bytes) return fail(CUBE_E_ARG, "NULL argument");
    int B = 0;
    cube_status s = check_params(params, &B);
    if (s != CUBE_OK) return s;
    cube_ctx c;
    init_geo(&c, params, B);
    size_t sec[5];
    *bytes = (int64_t)ckpt_layout(c.g, c.raw, params->id_bytes, sec);
    return CUBE_OK;
}

cube_status cube_checkpoint_save(cube_ctx* c, void* buf) {
    if (!c || !buf) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    const Geo& g = c->g;
    const int k = c->cur;
    size_t sec[5];
    ckpt_layout(g, c->raw, c->P.id_bytes, sec);
    CkptHeader h{};
    std::memcpy(h.magic, "CUBECKP1", 8);
    h.n_fine = g.N;
    h.ratio = g.R;
    h.n_particles = g.Np;
    h.x_bytes = c->raw ? 4 : g.nchi;
    h.v_bytes = c->raw ? 4 : g.nnu;
    h.id_bytes = c->P.id_bytes;
    h.brick = g.B;
    h.a = c->a;
    h.a_p = c->a_p;
    h.sigma = 0.0;
    if (!c->raw) CK(cudaMemcpyAsync(&h.sigma, c->codec[k].sigma, 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    char* b = (char*)buf;
    const size_t N = (size_t)g.Np, Ncc = (size_t)g.Ncc;
    CK(cudaMemcpyAsync(b, &h, sizeof(h), cudaMemcpyDefault, c->st));
    if (c->raw) {
        CK(cudaMemcpyAsync(b + sec[0], c->chi[0], 12 * N, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(b + sec[1], c->nu[0], 12 * N, cudaMemcpyDefault, c->st));
    } else {
        CK(cudaMemcpyAsync(b + sec[0], c->counts[k], 4 * Ncc, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(b + sec[1], c->vc[k], 12 * Ncc, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(b + sec[2], c->chi[k], 3 * N * g.nchi, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(b + sec[3], c->nu[k], 3 * N * g.nnu, cudaMemcpyDefault, c->st));
    }
    if (c->P.id_bytes) CK(cudaMemcpyAsync(b + sec[4], c->id[k], (size_t)c->P.id_bytes * N, cudaMemcpyDefault, c->st));
    return latched(c);
}

cube_status cube_checkpoint_load(cube_ctx* c, const void* buf) {
    if (!c || !buf) return fail(CUBE_E_ARG, "NULL argument");
    const Geo& g = c->g;
    CkptHeader h{};
    CK(cudaMemcpyAsync(&h, buf, sizeof(h), cudaMemcpyDefault, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (std::memcmp(h.magic, "CUBECKP1", 8) != 0) return fail(CUBE_E_ARG, "not a checkpoint (magic)");
    if (h.n_fine != g.N || h.ratio != g.R || h.n_particles != g.Np || h.brick != g.B ||
        h.x_bytes != (c->raw ? 4 : g.nchi) || h.v_bytes != (c->raw ? 4 : g.nnu) || h.id_bytes != c->P.id_bytes)
        return fail(CUBE_E_ARG, "checkpoint parameters differ from the context's");
    if (!(h.a > 0.0) || !(h.a_p > 0.0) || (!c->raw && !(h.sigma > 0.0)))
        return fail(CUBE_E_ARG, "checkpoint epochs or codec scale invalid");
    size_t sec[5];
    ckpt_layout(g, c->raw, c->P.id_bytes, sec);
    const char* b = (const char*)buf;
    const size_t N = (size_t)g.Np, Ncc = (size_t)g.Ncc;
    c->cur = 0;                          // a loaded store starts in buffer 0, as an encoded one
    const int k = c->cur;
    c->encoded = false;                  // until the whole store is in place
    if (c->raw) {
        CK(cudaMemcpyAsync(c->chi[0], b + sec[0], 12 * N, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(c->nu[0], b + sec[1], 12 * N, cudaMemcpyDefault, c->st));
    } else {
        CK(cudaMemcpyAsync(c->counts[k], b + sec[0], 4 * Ncc, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(c->vc[k], b + sec[1], 12 * Ncc, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(c->chi[k], b + sec[2], 3 * N * g.nchi, cudaMemcpyDefault, c->st));
        CK(cudaMemcpyAsync(c->nu[k], b + sec[3], 3 * N * g.nnu, cudaMemcpyDefault, c->st));
        exclusive_scan(c->counts[k], c->offsets[k], g.Ncc, c->scan_tmp, c->st);
        c->stage_sigma = h.sigma;
        CK(cudaMemcpyAsync(c->codec[k].sigma, &c->stage_sigma, 8, cudaMemcpyHostToDevice, c->st));
        launch_codec_tables(g.nulim, c->tanv, c->tanh_, c->codec[k], c->st);
        c->launches += 4 + 1;
    }
    if (c->P.id_bytes) CK(cudaMemcpyAsync(c->id[k], b + sec[4], (size_t)c->P.id_bytes * N, cudaMemcpyDefault, c->st));
    CK(cudaMemsetAsync(c->flags, 0, 4, c->st));
    CK(cudaMemsetAsync(c->maxmig, 0, 4, c->st));
    // the counts must add up to N_p in 64 bits, none above N_p (a sum that
    // only matches modulo 2^32 would pass a 32-bit check)
    unsigned long long tot[2] = {(unsigned long long)g.Np, 0ull};
    if (!c->raw) {
        count_totals(c->counts[k], g.Ncc, reinterpret_cast<unsigned long long*>(c->mom), c->st);
        c->launches += 1;
        CK(cudaMemcpyAsync(tot, c->mom, sizeof(tot), cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    c->phig_valid = false;
    c->a = h.a;
    c->a_p = h.a_p;
    c->steps = 0;
    c->version += 1;
    c->dbg_valid = false;
    c->timed = false;
    if (tot[0] != (unsigned long long)g.Np || tot[1] > (unsigned long long)g.Np)
        return fail(CUBE_E_ARG, "checkpoint cell counts do not add up to the particle count");
    c->encoded = true;
    return CUBE_OK;
}

cube_status cube_state_view(cube_ctx* c, cube_state* out) {
    if (!c || !out) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    const Geo& g = c->g;
    const int k = c->cur;
    out->n_coarse = g.Nc;
    out->brick = g.B;
    out->x_bytes = g.nchi;
    out->v_bytes = g.nnu;
    out->id_bytes = c->P.id_bytes;
    out->n_particles = g.Np;
    out->counts = c->raw ? nullptr : c->counts[k];
    out->offsets = c->raw ? nullptr : c->offsets[k];
    out->vc = c->raw ? nullptr : c->vc[k];
    out->chi = c->chi[k];
    out->nu = c->nu[k];
    out->id = c->id[k];
    out->sigma = 0.0;
    if (!c->raw) CK(cudaMemcpyAsync(&out->sigma, c->codec[k].sigma, 8, cudaMemcpyDeviceToHost, c->st));
    out->a = c->a;
    out->a_p = c->a_p;
    return latched(c);
}

cube_status cube_stats_get(cube_ctx* c, cube_stats* out) {
    if (!c || !out) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    const Geo& g = c->g;
    const int64_t launched = c->launches;          // before this call's own reduction
    if (c->raw) launch_raw_momentum(g, (const float*)c->nu[0], c->mom, c->st);
    else launch_store_sums(g, c->store(c->cur), c->codec[c->cur].dec, c->mom, c->st);
    c->launches += 1;
    long long m[4] = {0, 0, 0, g.Np};
    unsigned f = 0;
    int mig = 0;
    out->sigma = 0.0;
    CK(cudaMemcpyAsync(m, c->mom, (c->raw ? 3 : 4) * sizeof(long long), cudaMemcpyDeviceToHost, c->st));
    if (!c->raw) CK(cudaMemcpyAsync(&out->sigma, c->codec[c->cur].sigma, 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(&f, c->flags, 4, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(&mig, c->maxmig, 4, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    out->mass = (double)m[3] * particle_mass(g);
    for (int d = 0; d < 3; ++d) out->momentum[d] = (double)m[d] * std::ldexp(1.0, -24);
    out->a = c->a;
    out->a_p = c->a_p;
    out->steps = c->steps;
    out->max_migration = c->steps ? mig : 0;
    out->error_flags = f;
    float ms = 0.0f;
    if (c->timed) cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    out->last_step_ms = ms;
    out->kernel_launches = launched;
    out->features = c->tma ? 1u : 0u;
    return latched(c);
}

// unpadded N^3 copy of the mesh (density) or of the ghosted Phi
static cube_status mesh_out(cube_ctx* c, float* dst, bool phi) {
    const Geo& g = c->g;
    const size_t bytes = (size_t)g.N * g.N * g.N * 4;
    const bool host = !is_device_ptr(dst);
    float* d = dst;
    if (host) {
        void* p = nullptr;
        cube_status s = stage_bytes(c, bytes, &p);
        if (s != CUBE_OK) return s;
        d = (float*)p;
    }
    if (phi) launch_unpad_phig(c->phig, g.N, d, c->st);
    else launch_unpad(c->mesh, g.N, g.S, d, c->st);
    c->launches += 1;
    if (host) CK(cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, c->st));
    CK(cudaGetLastError());
    return latched(c);
}

cube_status cube_density(cube_ctx* c, float* rho) {
    if (!c || !rho) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    deposit(c);
    return mesh_out(c, rho, false);
}

cube_status cube_potential(cube_ctx* c, float* phi) {
    if (!c || !phi) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    const int saved = c->prof_max;
    c->prof_max = 0;                    // not a step: keep it out of the trace
    mesh_potential(c);
    c->phig_valid = true;
    c->prof_max = saved;
    return mesh_out(c, phi, true);
}

cube_status cube_keep_drifted(cube_ctx* c, int32_t enable) {
    if (!c) return fail(CUBE_E_ARG, "ctx is NULL");
    if (c->raw && enable) return fail(CUBE_E_STATE, "the uncompressed store has no re-sort to inspect");
    c->keep = enable != 0;
    if (!c->keep) {
        CK(cudaStreamSynchronize(c->st));
        cudaFree(c->dbg_cell);
        cudaFree(c->dbg_u);
        cudaFree(c->dbg_p);
        cudaFree(c->dbg_f);
        c->dbg_cell = nullptr;
        c->dbg_u = c->dbg_p = c->dbg_f = nullptr;
        c->dbg_valid = false;
    }
    return CUBE_OK;
}

cube_status cube_debug_drifted(cube_ctx* c, int32_t* cell_old, float* u_new, float* p, double* sigma_next) {
    if (!c || !cell_old || !u_new || !p) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->dbg_valid) return fail(CUBE_E_STATE, "no drifted state kept: enable cube_keep_drifted before the step");
    const size_t b = 12 * (size_t)c->g.Np;
    cube_status s;
    if ((s = to_user(c, cell_old, c->dbg_cell, b, !is_device_ptr(cell_old))) != CUBE_OK) return s;
    if ((s = to_user(c, u_new, c->dbg_u, b, !is_device_ptr(u_new))) != CUBE_OK) return s;
    if ((s = to_user(c, p, c->dbg_p, b, !is_device_ptr(p))) != CUBE_OK) return s;
    if (sigma_next) CK(cudaMemcpyAsync(sigma_next, c->codec[c->cur].sigma, 8, cudaMemcpyDeviceToHost, c->st));
    return latched(c);
}

cube_status cube_debug_force(cube_ctx* c, float* force) {
    if (!c || !force) return fail(CUBE_E_ARG, "NULL argument");
    if (!c->dbg_valid) return fail(CUBE_E_STATE, "no drifted state kept: enable cube_keep_drifted before the step");
    cube_status s = to_user(c, force, c->dbg_f, 12 * (size_t)c->g.Np, !is_device_ptr(force));
    if (s != CUBE_OK) return s;
    return latched(c);
}

cube_status cube_debug_velocity_tables(cube_ctx* c, int64_t* out2) {
    if (!c || !out2) return fail(CUBE_E_ARG, "NULL argument");
    if (c->raw || c->g.nnu != 2) return fail(CUBE_E_ARG, "the compact tables exist for 2-byte velocity codes only");
    if (!c->encoded) return fail(CUBE_E_STATE, "no store: call cube_encode first");
    launch_check_vel_tables(c->g.nulim, c->codec[c->cur], c->mom, c->st);
    c->launches += 2;
    long long h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, c->mom, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    out2[0] = h[0];
    out2[1] = h[1];
    return latched(c);
}

cube_status cube_profile(cube_ctx* c, int32_t max_steps) {
    if (!c) return fail(CUBE_E_ARG, "ctx is NULL");
    if (max_steps < 0 || max_steps > 100000) return fail(CUBE_E_ARG, "max_steps out of range");
    CK(cudaStreamSynchronize(c->st));
    const size_t need = (size_t)max_steps * (CUBE_PHASES + 1);
    while (c->prof_ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->prof_ev.push_back(e);
    }
    c->prof_max = max_steps;
    c->prof_steps = 0;
    return CUBE_OK;
}

cube_status cube_profile_read(cube_ctx* c, double* ms, int32_t* kernels, int32_t* nsteps) {
    if (!c || !ms) return fail(CUBE_E_ARG, "NULL argument");
    CK(cudaStreamSynchronize(c->st));
    for (int p = 0; p < CUBE_PHASES; ++p) {
        double t = 0.0;
        for (int s = 0; s < c->prof_steps; ++s) {
            float e = 0.0f;
            const size_t b = (size_t)s * (CUBE_PHASES + 1) + p;
            CK(cudaEventElapsedTime(&e, c->prof_ev[b], c->prof_ev[b + 1]));
            t += e;
        }
        ms[p] = t;
        if (kernels) kernels[p] = c->raw ? kPhaseKernelsRaw[p] : kPhaseKernels[p];
    }
    if (nsteps) *nsteps = c->prof_steps;
    return CUBE_OK;
}

const char* cube_phase_name(int32_t phase) {
    return (phase >= 0 && phase < CUBE_PHASES) ? kPhaseNames[phase] : "";
}

// ---------------------------------------------------------------- batches
// Simulations with the same geometry (mesh, particle count, codes, brick,
// cosmology and deconvolution; only the box may differ) stepped together:
// every member lives in one slab at a fixed stride, so each kernel of the
// step is launched once for all members (an extra grid dimension), with the
// members' own epochs, kick and drift factors from a per-member table.
struct cube_batch {
    std::vector<cube_ctx*> m;
    char* slab = nullptr;
    size_t stride = 0;
    cudaStream_t st = nullptr;
    CUtensorMap map{};                  // 4-D map (x, y, z, member) of the members' ghosted Phi
    bool tma = false;
    MemberStep* ms_dev = nullptr;       // [members]: the stepped members' table, one entry per grid slot
    MemberStep* ms_host = nullptr;      // pinned [members]
    std::vector<int> slots;             // the member of each slot of the last step
    MemberStep* solve_dev = nullptr;    // [members]: the member table of the last cube_batch_solve
    MemberStep* solve_host = nullptr;   // pinned [members]
    cudaEvent_t solve_copied = nullptr; // that table's upload has been read
    std::vector<int> solve_slots;
    std::vector<uint64_t> solved;       // per member: store version whose potential phig holds (0: none)
    // CUDA graphs of the two halves of a batch step, by (half, store parity, slots)
    struct Graph {
        int uses = 0;
        cudaGraphExec_t exec = nullptr;
    };
    std::map<int, Graph> graphs;
    bool graphs_on = false;             // meshes up to 256 (whose sweeps have batched instances)
    unsigned* vmax_host = nullptr;      // pinned [members]: largest |p| per member (float bits)
    cudaEvent_t ms_copied = nullptr;    // the last table upload has been read
    cudaEvent_t vmax_ready = nullptr;   // the maxima read-back has arrived
    bool vmax_pending = false;
    int64_t launches = 0;
};

cube_status cube_batch_destroy(cube_batch* b) {
    if (!b) return CUBE_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    for (cube_ctx* c : b->m) cube_destroy(c);
    if (b->slab) cudaFree(b->slab);
    if (b->ms_dev) cudaFree(b->ms_dev);
    if (b->ms_host) cudaFreeHost(b->ms_host);
    if (b->vmax_host) cudaFreeHost(b->vmax_host);
    if (b->ms_copied) cudaEventDestroy(b->ms_copied);
    if (b->solve_dev) cudaFree(b->solve_dev);
    if (b->solve_host) cudaFreeHost(b->solve_host);
    if (b->solve_copied) cudaEventDestroy(b->solve_copied);
    for (auto& kv : b->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (b->vmax_ready) cudaEventDestroy(b->vmax_ready);
    delete b;
    return CUBE_OK;
}

cube_status cube_batch_create(const cube_params* params, int32_t members, void* cuda_stream, cube_batch** out) {
    if (!out || !params) return fail(CUBE_E_ARG, "NULL argument");
    *out = nullptr;
    if (members < 1 || members > 4096) return fail(CUBE_E_ARG, "members must be in [1, 4096]");
    int B0 = 0;
    cube_status s = check_params(&params[0], &B0);
    if (s != CUBE_OK) return s;
    if (params[0].x_bytes == 4) return fail(CUBE_E_ARG, "batches hold compressed stores (x_bytes 1 or 2)");
    for (int i = 1; i < members; ++i) {
        const cube_params &p = params[i], &q = params[0];
        int B = 0;
        if ((s = check_params(&p, &B)) != CUBE_OK) return s;
        if (p.n_fine != q.n_fine || p.ratio != q.ratio || p.n_particles != q.n_particles || p.x_bytes != q.x_bytes ||
            p.v_bytes != q.v_bytes || p.id_bytes != q.id_bytes || p.omega_m != q.omega_m || p.omega_l != q.omega_l ||
            p.gradient != q.gradient || p.deconv_power != q.deconv_power || B != B0)
            return fail(CUBE_E_ARG, "batch members must share everything but the box");
    }
    cube_batch* b = new cube_batch();
    b->st = (cudaStream_t)cuda_stream;
    auto bad = [&](cudaError_t e, const char* what) -> cube_status {
        cube_batch_destroy(b);
        return fail(e == cudaErrorMemoryAllocation ? CUBE_E_NOMEM : CUBE_E_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    };
    {
        cube_ctx probe;
        init_geo(&probe, &params[0], B0);
        const size_t st_sz = state_layout(&probe, nullptr), wk_sz = work_layout(&probe, nullptr);
        b->stride = ((st_sz + 255) & ~(size_t)255) + ((wk_sz + 255) & ~(size_t)255);
    }
    cudaError_t e = cudaMalloc((void**)&b->slab, b->stride * (size_t)members);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->ms_dev, sizeof(MemberStep) * members);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->ms_host, sizeof(MemberStep) * members);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->vmax_host, sizeof(unsigned) * members);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ms_copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->vmax_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->solve_dev, sizeof(MemberStep) * members);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->solve_host, sizeof(MemberStep) * members);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->solve_copied, cudaEventDisableTiming);
    b->solved.assign(members, 0);
    b->graphs_on = params[0].n_fine <= 256;
    if (e != cudaSuccess) return bad(e, "device memory");
    for (int i = 0; i < members; ++i) {
        cube_ctx* c = nullptr;
        s = create_ctx(&params[i], cuda_stream, false, &c, b->slab + (size_t)i * b->stride);
        if (s != CUBE_OK) {
            const std::string msg = g_err;
            cube_batch_destroy(b);
            return fail(s, msg);
        }
        b->m.push_back(c);
    }
    b->tma = encode_phig_map(b->m[0]->g, b->m[0]->phig, members, b->stride, &b->map);
    *out = b;
    return CUBE_OK;
}

cube_status cube_batch_member(cube_batch* b, int32_t i, cube_ctx** out) {
    if (!b || !out) return fail(CUBE_E_ARG, "NULL argument");
    if (i < 0 || i >= (int)b->m.size()) return fail(CUBE_E_ARG, "member index out of range");
    *out = b->m[i];
    return CUBE_OK;
}

// every member's largest |p| into pinned memory (one copy: they lie one stride
// apart), enqueued, with an event marking its arrival
static cube_status batch_vmax_enqueue(cube_batch* b) {
    const int K = (int)b->m.size();
    bool same = true;
    for (int i = 0; i < K; ++i) {
        if (!b->m[i]->encoded) return fail(CUBE_E_STATE, "a member has no store: call cube_encode first");
        same = same && b->m[i]->cur == b->m[0]->cur;
    }
    if (same) {                                  // one launch over every member's store
        cube_ctx* c = b->m[0];
        launch_max_speed(c->g, c->store(c->cur), c->codec[c->cur].dec, c->vmax, b->st,
                         Batch{K, b->stride, nullptr, nullptr});
        b->launches += 2;
    } else {
        for (cube_ctx* c : b->m) {
            launch_max_speed(c->g, c->store(c->cur), c->codec[c->cur].dec, c->vmax, b->st);
            c->launches += 1;
        }
    }
    CK(cudaMemcpy2DAsync(b->vmax_host, sizeof(unsigned), b->m[0]->vmax, b->stride, sizeof(unsigned), K,
                         cudaMemcpyDeviceToHost, b->st));
    CK(cudaEventRecord(b->vmax_ready, b->st));
    b->vmax_pending = true;
    return CUBE_OK;
}

// the epochs from the read-back maxima (bisection on the host, as cube_next_epoch)
static cube_status batch_epochs(cube_batch* b, const double* a_max, double cells, double* a_to) {
    const int K = (int)b->m.size();
    for (int i = 0; i < K; ++i) {
        cube_ctx* c = b->m[i];
        if (!(a_max[i] > c->a)) {
            a_to[i] = c->a;
            continue;
        }
        float p;
        std::memcpy(&p, &b->vmax_host[i], 4);
        a_to[i] = epoch_limit(c, (double)p, a_max[i], cells);
        if (!(a_to[i] > c->a)) return fail(CUBE_E_ARG, "no step keeps a member's fastest particle within the limit");
    }
    return CUBE_OK;
}

cube_status cube_batch_next_epochs(cube_batch* b, const double* a_max, double cells, double* a_to) {
    if (!b || !a_max || !a_to) return fail(CUBE_E_ARG, "NULL argument");
    if (!(cells > 0.0 && cells <= 1.0)) return fail(CUBE_E_ARG, "cells must be in (0, 1]");
    cube_status s = batch_vmax_enqueue(b);
    if (s != CUBE_OK) return s;
    CK(cudaEventSynchronize(b->vmax_ready));
    b->vmax_pending = false;
    return batch_epochs(b, a_max, cells, a_to);
}

cube_status cube_batch_epochs_enqueue(cube_batch* b) {
    if (!b) return fail(CUBE_E_ARG, "NULL argument");
    return batch_vmax_enqueue(b);
}

cube_status cube_batch_epochs_poll(cube_batch* b, const double* a_max, double cells, double* a_to, int32_t* ready) {
    if (!b || !a_max || !a_to || !ready) return fail(CUBE_E_ARG, "NULL argument");
    if (!(cells > 0.0 && cells <= 1.0)) return fail(CUBE_E_ARG, "cells must be in (0, 1]");
    *ready = 0;
    if (!b->vmax_pending) return fail(CUBE_E_STATE, "no read-back enqueued: call cube_batch_epochs_enqueue first");
    const cudaError_t q = cudaEventQuery(b->vmax_ready);
    if (q == cudaErrorNotReady) return CUBE_OK;
    if (q != cudaSuccess) return fail(CUBE_E_CUDA, cudaGetErrorString(q));
    b->vmax_pending = false;
    *ready = 1;
    return batch_epochs(b, a_max, cells, a_to);
}

// One half of a batch step from a CUDA graph.  The launch sequence of a half
// depends only on the key (which half, the store parity, the number of
// slots): per-member values reach the kernels through the device table.  The
// first use of a key launches directly (which also sets the kernels'
// attributes), the second captures the sequence and instantiates it, later
// ones replay it.  Any capture error turns graphs off for the batch and
// launches directly.
static cube_status batch_graph(cube_batch* b, int key, const std::function<void()>& enqueue) {
    if (!b->graphs_on) {
        enqueue();
        return CUBE_OK;
    }
    cube_batch::Graph& e = b->graphs[key];
    if (e.exec) {
        CK(cudaGraphLaunch(e.exec, b->st));
        return CUBE_OK;
    }
    if (e.uses++ == 0) {
        enqueue();
        return CUBE_OK;
    }
    cudaGraph_t gr = nullptr;
    cudaError_t err = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        enqueue();
        err = cudaStreamEndCapture(b->st, &gr);
        if (err == cudaSuccess) err = cudaGraphInstantiate(&e.exec, gr, 0);
        if (gr) cudaGraphDestroy(gr);
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        e.exec = nullptr;
        b->graphs_on = false;
        enqueue();
        return CUBE_OK;
    }
    CK(cudaGraphLaunch(e.exec, b->st));
    return CUBE_OK;
}

// deposit and Poisson solve of the listed members' current stores into their
// ghosted potentials (the mesh half of a step), one launch per kernel
static cube_status batch_solve(cube_batch* b, const std::vector<int>& members) {
    if (members.empty()) return CUBE_OK;
    CK(cudaEventSynchronize(b->solve_copied));                      // the previous table has been read
    b->solve_slots = members;
    for (size_t j = 0; j < members.size(); ++j)
        b->solve_host[j] = MemberStep{0.0f, 0.0f, 1.0, 1, members[j]};
    const int n = (int)members.size();
    CK(cudaMemcpyAsync(b->solve_dev, b->solve_host, sizeof(MemberStep) * n, cudaMemcpyHostToDevice, b->st));
    CK(cudaEventRecord(b->solve_copied, b->st));
    cube_ctx* c0 = b->m[0];
    const Geo& g = c0->g;
    const int k = b->m[members[0]]->cur;
    const Batch bt{n, b->stride, b->solve_dev, b->solve_slots.data()};
    const float g0 = (float)(-1.5 * c0->P.omega_m / std::pow((double)g.N, 3));
    cube_status gs = batch_graph(b, (0 * 2 + k) * 8192 + n, [&] {
        launch_deposit(g, c0->store(k), c0->mesh, particle_mass(g) * std::ldexp(1.0, -3 * g.sbits), b->st, bt);
        fft_x_r2c(c0->fft, c0->mesh, g.S, b->st, bt);
        fft_y(c0->fft, c0->mesh, g.S, false, b->st, bt);
        fft_z(c0->fft, c0->mesh, g.S, g0, true, b->st, bt);
        fft_y(c0->fft, c0->mesh, g.S, true, b->st, bt);
        fft_x_c2r(c0->fft, c0->mesh, g.S, c0->phig, b->st, bt);
    });
    if (gs != CUBE_OK) return gs;
    b->launches += 6;
    CK(cudaGetLastError());
    for (int i : members) {
        b->solved[i] = b->m[i]->version;
        b->m[i]->phig_valid = true;
    }
    return CUBE_OK;
}

cube_status cube_batch_solve(cube_batch* b, const int32_t* stepping) {
    if (!b || !stepping) return fail(CUBE_E_ARG, "NULL argument");
    std::vector<int> list;
    int cur = -1;
    for (int i = 0; i < (int)b->m.size(); ++i) {
        if (!stepping[i]) continue;
        cube_ctx* c = b->m[i];
        if (!c->encoded) return fail(CUBE_E_STATE, "a member has no store: call cube_encode first");
        if (cur >= 0 && c->cur != cur)
            return fail(CUBE_E_STATE, "members solved together must have taken the same number of steps");
        cur = c->cur;
        if (b->solved[i] != c->version) list.push_back(i);
    }
    return batch_solve(b, list);
}

cube_status cube_batch_step(cube_batch* b, const double* a_from, const double* a_to) {
    if (!b || !a_from || !a_to) return fail(CUBE_E_ARG, "NULL argument");
    const int K = (int)b->m.size();
    int cur = -1, nact = 0;
    for (int i = 0; i < K; ++i) {
        cube_ctx* c = b->m[i];
        if (!(a_to[i] > a_from[i])) continue;                       // sits this step out
        if (!c->encoded) return fail(CUBE_E_STATE, "a member has no store: call cube_encode first");
        if (std::fabs(a_from[i] - c->a) > 1e-12 * std::max(1.0, std::fabs(a_from[i])))
            return fail(CUBE_E_STATE, "a member's a_from differs from its store's epoch");
        if (cur >= 0 && c->cur != cur)
            return fail(CUBE_E_STATE, "members stepped together must have taken the same number of steps "
                                      "(a member that sat a step out continues with cube_pm_step)");
        cur = c->cur;
        ++nact;
    }
    if (!nact) return CUBE_OK;
    CK(cudaEventSynchronize(b->ms_copied));                         // the previous table has been read
    // one grid slot per stepped member: members that sit the step out get no CTAs
    b->slots.clear();
    for (int i = 0; i < K; ++i) {
        if (!(a_to[i] > a_from[i])) continue;
        cube_ctx* c = b->m[i];
        MemberStep& ms = b->ms_host[b->slots.size()];
        const double a_mid = 0.5 * (a_from[i] + a_to[i]);
        ms.kick = (float)c->cosmo.kick(c->a_p, a_mid);
        ms.dc = (float)(c->cosmo.drift(a_from[i], a_to[i]) / c->g.R);
        ms.ratio = c->cosmo.g(a_to[i]) / c->cosmo.g(a_from[i]);
        ms.active = 1;
        ms.member = i;
        b->slots.push_back(i);
    }
    CK(cudaMemcpyAsync(b->ms_dev, b->ms_host, sizeof(MemberStep) * nact, cudaMemcpyHostToDevice, b->st));
    CK(cudaEventRecord(b->ms_copied, b->st));
    cube_ctx* c0 = b->m[0];
    const Geo& g = c0->g;
    const int k = cur, kn = 1 - cur;
    // the potential of every stepped member's current store: solved ahead
    // (cube_batch_solve) or now
    std::vector<int> need;
    for (int i : b->slots)
        if (b->solved[i] != b->m[i]->version) need.push_back(i);
    cube_status ss = batch_solve(b, need);
    if (ss != CUBE_OK) return ss;
    const Batch bt{nact, b->stride, b->ms_dev, b->slots.data()};
    const StepScratch w{c0->counts[kn], c0->vsum, c0->ghost, c0->part, c0->flags, c0->maxmig, c0->maxmig + 1};
    const DriftDebug nodbg{nullptr, nullptr, nullptr, nullptr};
    cube_status gs = batch_graph(b, (1 * 2 + k) * 8192 + nact, [&] {
        launch_batch_clear(g, c0->vsum, c0->maxmig, b->st, bt);
        launch_passA(g, c0->store(k), c0->phig, b->tma ? &b->map : nullptr, c0->codec[k], 0.0f, 0.0f, w, nodbg,
                     b->st, bt);
        launch_sigma_finalize(c0->part, g.nbricks, 3.0 * (double)g.Np, 1.0, 0.0, c0->codec[kn].sigma, b->st, bt);
        launch_codec_tables(g.nulim, c0->tanv, c0->tanh_, c0->codec[kn], b->st, bt);
        exclusive_scan(c0->ghost, c0->ghost, (int64_t)g.nbricks * (g.Bh * g.Bh * g.Bh), c0->scan_tmp, b->st, bt);
        launch_cells(g, w, c0->offsets[kn], c0->vc[kn], b->st, bt);
        launch_passB(g, c0->store(k), c0->store(kn), c0->codec[k], c0->codec[kn], 0.0f, w, b->st, bt);
    });
    if (gs != CUBE_OK) return gs;
    b->launches += 1 + 1 + 2 + 4 + 1 + 1;
    CK(cudaGetLastError());
    for (int i = 0; i < K; ++i) {
        cube_ctx* c = b->m[i];
        if (!(a_to[i] > a_from[i])) continue;
        c->cur = kn;
        c->a_p = 0.5 * (a_from[i] + a_to[i]);
        c->a = a_to[i];
        c->steps += 1;
        c->version += 1;
        c->phig_valid = true;
        c->dbg_valid = false;
        c->timed = false;
    }
    return CUBE_OK;
}

cube_status cube_batch_launches(cube_batch* b, int64_t* launches) {
    if (!b || !launches) return fail(CUBE_E_ARG, "NULL argument");
    *launches = b->launches;
    return CUBE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- hooks for the server (serve.cu)
namespace cube {

cube_status served_sizes(const cube_params* p, size_t* state, size_t* work) {
    int B = 0;
    cube_status s = check_params(p, &B);
    if (s != CUBE_OK) return s;
    cube_ctx c;
    init_geo(&c, p, B);
    *state = state_layout(&c, nullptr);
    *work = work_layout(&c, nullptr);
    return CUBE_OK;
}

cube_status served_create(const cube_params* p, cudaStream_t st, cube_ctx** out) {
    return create_ctx(p, st, true, out);
}

cube_status served_bind(cube_ctx* c, char* work) {
    if (!work) return fail(CUBE_E_NOMEM, "the request's stream has no work area");
    if (c->work_base == work) return CUBE_OK;
    c->work_base = work;
    work_layout(c, work);
    c->tma = encode_phig_map(c);
    return CUBE_OK;
}

cube_status served_encode(cube_ctx* c, const float* pos, const float* vel, const uint32_t* id, double a,
                          double sigma) {
    return encode_impl(c, pos, vel, id, a, sigma, false);
}

cube_status served_finish(cube_ctx* c, int32_t n_bins, double* pk3, unsigned* flags2) {
    cube_status s = pk_enqueue(c, n_bins, pk3, pk3 + n_bins, pk3 + 2 * n_bins);
    if (s != CUBE_OK) return s;
    CK(cudaMemcpyAsync(flags2, c->flags, 4, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(flags2 + 1, c->maxmig, 4, cudaMemcpyDeviceToHost, c->st));
    return CUBE_OK;
}

cube_status served_flags_status(unsigned flags) { return flags_status(flags); }

// largest |p| of the store into pinned host memory (float bits), enqueued
cube_status served_vmax_enqueue(cube_ctx* c, unsigned* pinned_bits) {
    const Geo& g = c->g;
    if (c->raw) launch_raw_max_speed(g, (const float*)c->nu[0], c->vmax, c->st);
    else launch_max_speed(g, c->store(c->cur), c->codec[c->cur].dec, c->vmax, c->st);
    c->launches += 1;
    CK(cudaMemcpyAsync(pinned_bits, c->vmax, 4, cudaMemcpyDeviceToHost, c->st));
    return CUBE_OK;
}

double served_epoch_limit(cube_ctx* c, double p_max, double a_max, double cells) {
    return epoch_limit(c, p_max, a_max, cells);
}

double served_epoch(cube_ctx* c) { return c->a; }

cube_status served_fail(cube_status s, const char* msg) { return fail(s, msg); }

}  // namespace cube
