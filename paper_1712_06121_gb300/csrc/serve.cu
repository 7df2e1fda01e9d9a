// Continuous-batching server: many independent simulations on one GPU.
// See include/cube.h (serving) for the contract.
//
// A request's life: QUEUED (host arrays referenced, nothing on the device)
// -> admitted in arrival order once its state slab and its stream's work
// area fit the budget -> RUNNING (encode, then one step after another, at
// most kDepth steps in flight, interleaved with the other requests of its
// stream) -> final P(k) and error flags copied into pinned host memory ->
// DONE when that copy's event has completed.  The state slab stays resident
// until cube_server_release.  The host never waits on the GPU in pump().
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "cube.h"
#include "kernels.h"

namespace cube {
cube_status served_sizes(const cube_params* p, size_t* state, size_t* work);
cube_status served_create(const cube_params* p, cudaStream_t st, cube_ctx** out);
cube_status served_bind(cube_ctx* c, char* work);
cube_status served_encode(cube_ctx* c, const float* pos, const float* vel, const uint32_t* id, double a,
                          double sigma);
cube_status served_finish(cube_ctx* c, int32_t n_bins, double* pk3, unsigned* flags2);
cube_status served_flags_status(unsigned flags);
cube_status served_fail(cube_status s, const char* msg);
cube_status served_vmax_enqueue(cube_ctx* c, unsigned* pinned_bits);
double served_epoch_limit(cube_ctx* c, double p_max, double a_max, double cells);
double served_epoch(cube_ctx* c);
}  // namespace cube

using namespace cube;

namespace {

constexpr int kDepth = 2;      // steps of one request in flight

struct Request {
    int64_t ticket = 0;
    cube_params prm{};
    const float* pos = nullptr;
    const float* vel = nullptr;
    const uint32_t* id = nullptr;
    double sigma = 0.0;
    std::vector<double> epochs;           // fixed steps, or the waypoints of adaptive ones
    double cells = 0.0;                   // > 0: each step cut so the fastest particle drifts <= cells
    int n_bins = 0;
    int waypoint = 1;                     // adaptive: next epochs[] index to reach
    bool vmax_pending = false;            // adaptive: the max-speed copy of the current state is queued
    cudaEvent_t vmax_ev = nullptr;
    size_t state_bytes = 0, work_bytes = 0;
    int state = CUBE_REQ_QUEUED;
    int next = 0;                         // steps enqueued
    int slot = -1;
    bool finishing = false;               // P(k) enqueued
    cube_ctx* ctx = nullptr;
    std::deque<cudaEvent_t> inflight;     // one event per enqueued step
    cudaEvent_t done = nullptr;
    double* pk = nullptr;                 // pinned [3][n_bins]
    unsigned* flags = nullptr;            // pinned {error flags, max migration, max |p| bits}
    double t_submit = -1.0, t_admit = -1.0, t_done = -1.0;
    cube_status err = CUBE_OK;
};

struct Slot {
    cudaStream_t st = nullptr;
    char* work = nullptr;                 // shared work area of the stream's requests
    size_t bytes = 0;
    int running = 0;
};

#define SCK(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return served_fail(e_ == cudaErrorMemoryAllocation ? CUBE_E_NOMEM : CUBE_E_CUDA, \
                               (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
    } while (0)

}  // namespace

struct cube_server {
    int64_t budget = 0;
    int64_t used = 0;                     // resident states + work areas
    int max_running = 1;
    std::vector<Slot> slots;
    std::deque<Request*> queue;
    std::vector<Request*> running;
    std::map<int64_t, Request*> reqs;
    std::vector<cudaEvent_t> spare;       // recycled step events
    int64_t next_ticket = 1;
    int inject_alloc_failures = 0;        // test hook: work-area allocations to refuse
    int policy = CUBE_ADMIT_FIFO;         // which queued request is admitted next
    std::chrono::steady_clock::time_point t0;

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }

    cudaEvent_t event() {
        if (!spare.empty()) {
            cudaEvent_t e = spare.back();
            spare.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }
};

namespace {

void fail_request(cube_server* s, Request* r, cube_status err) {
    r->err = err;
    r->state = CUBE_REQ_FAILED;
    r->t_done = s->now();
}

// retire finished steps; enqueue steps up to kDepth in flight; then P(k)
cube_status advance(cube_server* s, Request* r) {
    Slot& sl = s->slots[r->slot];
    while (!r->inflight.empty()) {
        const cudaError_t q = cudaEventQuery(r->inflight.front());
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return served_fail(CUBE_E_CUDA, cudaGetErrorString(q));
        s->spare.push_back(r->inflight.front());
        r->inflight.pop_front();
    }
    const int n_steps = (int)r->epochs.size() - 1;
    if (r->cells > 0.0) {                 // adaptive: one step per max-speed read-back
        if (r->finishing) goto finish;
        if (!r->vmax_pending) {
            cube_status st = served_bind(r->ctx, sl.work);
            if (st == CUBE_OK) st = served_vmax_enqueue(r->ctx, &r->flags[2]);
            if (st != CUBE_OK) {
                fail_request(s, r, st);
                return CUBE_OK;
            }
            if (!r->vmax_ev) SCK(cudaEventCreateWithFlags(&r->vmax_ev, cudaEventDisableTiming));
            SCK(cudaEventRecord(r->vmax_ev, sl.st));
            r->vmax_pending = true;
            return CUBE_OK;
        }
        const cudaError_t q = cudaEventQuery(r->vmax_ev);
        if (q == cudaErrorNotReady) return CUBE_OK;
        if (q != cudaSuccess) return served_fail(CUBE_E_CUDA, cudaGetErrorString(q));
        r->vmax_pending = false;
        const double a = served_epoch(r->ctx);
        if (a < r->epochs[n_steps]) {
            float p;
            std::memcpy(&p, &r->flags[2], 4);
            const double a_to = served_epoch_limit(r->ctx, (double)p, r->epochs[r->waypoint], r->cells);
            if (!(a_to > a)) {
                fail_request(s, r, served_fail(CUBE_E_ARG, "no step keeps the fastest particle within the limit"));
                return CUBE_OK;
            }
            cube_status st = served_bind(r->ctx, sl.work);
            if (st == CUBE_OK) st = cube_pm_step(r->ctx, a, a_to);
            if (st != CUBE_OK) {
                fail_request(s, r, st);
                return CUBE_OK;
            }
            ++r->next;
            if (a_to >= r->epochs[r->waypoint]) ++r->waypoint;
            if (a_to < r->epochs[n_steps]) return advance(s, r);     // queue the next read-back
        }
        r->waypoint = n_steps + 1;
    }
    while (r->cells <= 0.0 && r->next < n_steps && (int)r->inflight.size() < kDepth) {
        cube_status st = served_bind(r->ctx, sl.work);
        if (st == CUBE_OK) st = cube_pm_step(r->ctx, r->epochs[r->next], r->epochs[r->next + 1]);
        if (st != CUBE_OK) {
            fail_request(s, r, st);
            return CUBE_OK;
        }
        cudaEvent_t e = s->event();
        SCK(cudaEventRecord(e, sl.st));
        r->inflight.push_back(e);
        ++r->next;
    }
    if ((r->cells > 0.0 ? r->waypoint > n_steps : r->next == n_steps) && !r->finishing) {
        cube_status st = served_bind(r->ctx, sl.work);
        if (st == CUBE_OK) st = served_finish(r->ctx, r->n_bins, r->pk, r->flags);
        if (st != CUBE_OK) {
            fail_request(s, r, st);
            return CUBE_OK;
        }
        SCK(cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming));
        SCK(cudaEventRecord(r->done, sl.st));
        r->finishing = true;
    }
finish:
    if (r->finishing) {
        const cudaError_t q = cudaEventQuery(r->done);
        if (q == cudaSuccess) {
            r->t_done = s->now();
            r->err = served_flags_status(r->flags[0]);
            r->state = r->err == CUBE_OK ? CUBE_REQ_DONE : CUBE_REQ_FAILED;
        } else if (q != cudaErrorNotReady) {
            return served_fail(CUBE_E_CUDA, cudaGetErrorString(q));
        }
    }
    return CUBE_OK;
}

// remaining work of a queued request: particles x scheduled steps
double request_work(const Request* r) {
    return (double)r->prm.n_particles * (double)(r->epochs.size() - 1);
}

cube_status admit(cube_server* s) {
    while (!s->queue.empty() && (int)s->running.size() < s->max_running) {
        // FIFO: the oldest request; shortest first: the least remaining work
        // (ties: the oldest).  The chosen request waits for memory; nothing
        // behind it overtakes it.
        auto pick = s->queue.begin();
        if (s->policy == CUBE_ADMIT_SHORTEST)
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
                if (request_work(*it) < request_work(*pick)) pick = it;
        Request* r = *pick;
        // the stream with the fewest running requests whose work area fits
        // the request (or can grow within the budget); ties: no growth, then
        // the lowest index
        int k = -1;
        int64_t grow = 0;
        for (int i = 0; i < (int)s->slots.size(); ++i) {
            const Slot& c = s->slots[i];
            const int64_t g = r->work_bytes > c.bytes ? (int64_t)(r->work_bytes - c.bytes) : 0;
            if (s->used + (int64_t)r->state_bytes + g > s->budget) continue;
            if (k < 0 || c.running < s->slots[k].running || (c.running == s->slots[k].running && g == 0 && grow > 0)) {
                k = i;
                grow = g;
            }
        }
        if (k < 0) break;                 // in arrival order: wait for memory
        Slot& sl = s->slots[k];
        if (grow) {
            // the larger area is allocated before the old one is released, so
            // the stream's running requests keep a valid work area whatever
            // happens; without memory, this request alone fails
            char* fresh = nullptr;
            cudaError_t e = cudaErrorMemoryAllocation;
            if (s->inject_alloc_failures > 0) --s->inject_alloc_failures;
            else e = cudaMallocAsync((void**)&fresh, r->work_bytes, sl.st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s->queue.erase(pick);
                if (e != cudaErrorMemoryAllocation) {
                    fail_request(s, r, CUBE_E_CUDA);
                    return served_fail(CUBE_E_CUDA, cudaGetErrorString(e));
                }
                fail_request(s, r, served_fail(CUBE_E_NOMEM, "no device memory for the stream's larger work area"));
                continue;
            }
            if (sl.work) SCK(cudaFreeAsync(sl.work, sl.st));   // stream-ordered: its last user runs first
            s->used += (int64_t)r->work_bytes - (int64_t)sl.bytes;
            sl.work = fresh;
            sl.bytes = r->work_bytes;
        }
        s->queue.erase(pick);
        r->slot = k;
        r->t_admit = s->now();
        cube_status st = served_create(&r->prm, sl.st, &r->ctx);
        if (st == CUBE_OK) {
            s->used += (int64_t)r->state_bytes;
            st = served_bind(r->ctx, sl.work);
            if (st == CUBE_OK) st = served_encode(r->ctx, r->pos, r->vel, r->id, r->epochs[0], r->sigma);
        }
        if (st != CUBE_OK) {
            fail_request(s, r, st);
            continue;
        }
        r->state = CUBE_REQ_RUNNING;
        ++sl.running;
        s->running.push_back(r);
    }
    return CUBE_OK;
}

Request* find(cube_server* s, int64_t t) {
    auto it = s->reqs.find(t);
    return it == s->reqs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

cube_status cube_server_sizes(const cube_params* params, int64_t* state_bytes, int64_t* work_bytes) {
    if (!state_bytes || !work_bytes) return served_fail(CUBE_E_ARG, "outputs required");
    size_t a = 0, b = 0;
    cube_status s = served_sizes(params, &a, &b);
    if (s != CUBE_OK) return s;
    *state_bytes = (int64_t)a;
    *work_bytes = (int64_t)b;
    return CUBE_OK;
}

cube_status cube_server_create(int64_t budget_bytes, int32_t n_streams, int32_t max_running, cube_server** out) {
    if (!out) return served_fail(CUBE_E_ARG, "out is NULL");
    *out = nullptr;
    if (budget_bytes <= 0 || n_streams < 1 || n_streams > 64 || max_running < 1)
        return served_fail(CUBE_E_ARG, "budget > 0, n_streams in [1, 64], max_running >= 1");
    cube_server* s = new cube_server();
    s->budget = budget_bytes;
    s->max_running = max_running;
    s->t0 = std::chrono::steady_clock::now();
    s->slots.resize(n_streams);
    for (Slot& sl : s->slots) {
        const cudaError_t e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cube_server_destroy(s);
            return served_fail(CUBE_E_CUDA, cudaGetErrorString(e));
        }
    }
    *out = s;
    return CUBE_OK;
}

cube_status cube_server_destroy(cube_server* s) {
    if (!s) return CUBE_OK;
    for (Slot& sl : s->slots)
        if (sl.st) cudaStreamSynchronize(sl.st);
    for (auto& kv : s->reqs) {
        Request* r = kv.second;
        if (r->ctx) cube_destroy(r->ctx);
        for (cudaEvent_t e : r->inflight) cudaEventDestroy(e);
        if (r->done) cudaEventDestroy(r->done);
        if (r->vmax_ev) cudaEventDestroy(r->vmax_ev);
        if (r->pk) cudaFreeHost(r->pk);
        delete r;
    }
    for (cudaEvent_t e : s->spare) cudaEventDestroy(e);
    for (Slot& sl : s->slots) {
        if (sl.work) cudaFreeAsync(sl.work, sl.st);
        if (sl.st) {
            cudaStreamSynchronize(sl.st);
            cudaStreamDestroy(sl.st);
        }
    }
    delete s;
    return CUBE_OK;
}

cube_status cube_server_submit(cube_server* s, const cube_params* params, const float* pos, const float* vel,
                               const uint32_t* id, double sigma, const double* epochs, int32_t n_steps,
                               double max_drift_cells, int32_t n_bins, int64_t* ticket) {
    if (!s || !params || !pos || !vel || !epochs || !ticket) return served_fail(CUBE_E_ARG, "NULL argument");
    if (!(max_drift_cells >= 0.0 && max_drift_cells <= 1.0))
        return served_fail(CUBE_E_ARG, "max_drift_cells must be 0 (fixed steps) or in (0, 1]");
    if (n_steps < 1) return served_fail(CUBE_E_ARG, "n_steps must be >= 1");
    if (n_bins < 1 || n_bins > 2048) return served_fail(CUBE_E_ARG, "n_bins in [1, 2048]");
    if (!(epochs[0] > 0.0)) return served_fail(CUBE_E_ARG, "epochs[0] must be > 0");
    for (int i = 0; i < n_steps; ++i)
        if (!(epochs[i + 1] > epochs[i])) return served_fail(CUBE_E_ARG, "epochs must increase");
    size_t sb = 0, wb = 0;
    cube_status st = served_sizes(params, &sb, &wb);
    if (st != CUBE_OK) return st;
    if ((int64_t)(sb + wb) > s->budget) return served_fail(CUBE_E_NOMEM, "the request alone exceeds the budget");
    Request* r = new Request();
    const size_t pinned = (size_t)3 * n_bins * 8 + 3 * sizeof(unsigned);
    if (cudaMallocHost((void**)&r->pk, pinned) != cudaSuccess) {
        delete r;
        return served_fail(CUBE_E_NOMEM, "pinned result memory");
    }
    r->flags = reinterpret_cast<unsigned*>(r->pk + 3 * (size_t)n_bins);
    r->flags[0] = r->flags[1] = r->flags[2] = 0;
    r->ticket = s->next_ticket++;
    r->prm = *params;
    r->pos = pos;
    r->vel = vel;
    r->id = id;
    r->sigma = sigma;
    r->epochs.assign(epochs, epochs + n_steps + 1);
    r->cells = max_drift_cells;
    r->n_bins = n_bins;
    r->state_bytes = sb;
    r->work_bytes = wb;
    r->t_submit = s->now();
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    return CUBE_OK;
}

cube_status cube_server_pump(cube_server* s, int32_t* n_running, int32_t* n_queued) {
    if (!s) return served_fail(CUBE_E_ARG, "server is NULL");
    for (Request* r : s->running) {
        cube_status st = advance(s, r);
        if (st != CUBE_OK) return st;
    }
    // finished requests leave the running set (their state stays resident)
    for (size_t i = 0; i < s->running.size();) {
        Request* r = s->running[i];
        if (r->state == CUBE_REQ_DONE || r->state == CUBE_REQ_FAILED) {
            --s->slots[r->slot].running;
            s->running.erase(s->running.begin() + (long)i);
        } else {
            ++i;
        }
    }
    cube_status st = admit(s);
    if (st != CUBE_OK) return st;
    for (Request* r : s->running)          // first steps of the newly admitted
        if (r->next == 0 && (st = advance(s, r)) != CUBE_OK) return st;
    if (n_running) *n_running = (int32_t)s->running.size();
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    return CUBE_OK;
}

cube_status cube_server_drain(cube_server* s) {
    if (!s) return served_fail(CUBE_E_ARG, "server is NULL");
    int32_t nr = 0, nq = 0;
    do {
        cube_status st = cube_server_pump(s, &nr, &nq);
        if (st != CUBE_OK) return st;
        if (nr + nq) std::this_thread::sleep_for(std::chrono::microseconds(50));
    } while (nr + nq);
    return CUBE_OK;
}

cube_status cube_server_info(cube_server* s, int64_t ticket, cube_request_info* out) {
    if (!s || !out) return served_fail(CUBE_E_ARG, "NULL argument");
    Request* r = find(s, ticket);
    if (!r) return served_fail(CUBE_E_ARG, "unknown ticket");
    out->state = r->state;
    out->steps_enqueued = r->next;
    out->n_steps = (int32_t)r->epochs.size() - 1;
    out->max_migration = r->state == CUBE_REQ_DONE || r->state == CUBE_REQ_FAILED ? (int32_t)r->flags[1] : 0;
    out->t_submit = r->t_submit;
    out->t_admit = r->t_admit;
    out->t_done = r->t_done;
    out->state_bytes = (int64_t)r->state_bytes;
    out->error = r->err;
    return CUBE_OK;
}

cube_status cube_server_result(cube_server* s, int64_t ticket, double* k, double* pk, double* nmodes) {
    if (!s || !k || !pk || !nmodes) return served_fail(CUBE_E_ARG, "NULL argument");
    Request* r = find(s, ticket);
    if (!r) return served_fail(CUBE_E_ARG, "unknown ticket");
    if (r->state != CUBE_REQ_DONE) return served_fail(CUBE_E_STATE, "request not done");
    const size_t b = (size_t)r->n_bins * 8;
    SCK(cudaMemcpy(k, r->pk, b, cudaMemcpyDefault));
    SCK(cudaMemcpy(pk, r->pk + r->n_bins, b, cudaMemcpyDefault));
    SCK(cudaMemcpy(nmodes, r->pk + 2 * r->n_bins, b, cudaMemcpyDefault));
    return CUBE_OK;
}

cube_status cube_server_decode(cube_server* s, int64_t ticket, float* pos, float* vel, uint32_t* id) {
    if (!s) return served_fail(CUBE_E_ARG, "server is NULL");
    Request* r = find(s, ticket);
    if (!r) return served_fail(CUBE_E_ARG, "unknown ticket");
    if (r->state != CUBE_REQ_DONE) return served_fail(CUBE_E_STATE, "request not done");
    cube_status st = served_bind(r->ctx, s->slots[r->slot].work);
    if (st != CUBE_OK) return st;
    return cube_decode(r->ctx, pos, vel, id);
}

cube_status cube_server_release(cube_server* s, int64_t ticket) {
    if (!s) return served_fail(CUBE_E_ARG, "server is NULL");
    Request* r = find(s, ticket);
    if (!r) return served_fail(CUBE_E_ARG, "unknown ticket");
    if (r->state != CUBE_REQ_DONE && r->state != CUBE_REQ_FAILED)
        return served_fail(CUBE_E_STATE, "request still queued or running");
    if (r->ctx) {
        cube_destroy(r->ctx);             // stream-ordered free of the state slab
        s->used -= (int64_t)r->state_bytes;
    }
    for (cudaEvent_t e : r->inflight) s->spare.push_back(e);
    if (r->done) cudaEventDestroy(r->done);
    if (r->vmax_ev) cudaEventDestroy(r->vmax_ev);
    if (r->pk) cudaFreeHost(r->pk);
    s->reqs.erase(ticket);
    delete r;
    return CUBE_OK;
}

cube_status cube_server_set_policy(cube_server* s, int32_t policy) {
    if (!s || (policy != CUBE_ADMIT_FIFO && policy != CUBE_ADMIT_SHORTEST))
        return served_fail(CUBE_E_ARG, "server is NULL or the policy is unknown");
    s->policy = policy;
    return CUBE_OK;
}

cube_status cube_server_inject_alloc_failures(cube_server* s, int32_t n) {
    if (!s || n < 0) return served_fail(CUBE_E_ARG, "server is NULL or n < 0");
    s->inject_alloc_failures = n;
    return CUBE_OK;
}

cube_status cube_server_bytes(cube_server* s, int64_t* bytes_in_use) {
    if (!s || !bytes_in_use) return served_fail(CUBE_E_ARG, "NULL argument");
    *bytes_in_use = s->used;
    return CUBE_OK;
}

}  // extern "C"
