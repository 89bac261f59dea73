// Serving layer: a queue of independent trajectories admitted by device memory
// and stepped together in one batched graph (continuous batching).  Built only
// on the public context and batch calls; host code.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "mix.h"

namespace {

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Request {
    int64_t id = 0;
    int state = MIX_REQ_QUEUED;
    int status = MIX_OK;
    mix_ctx* ctx = nullptr;
    int64_t n = 0;
    size_t ws_bytes = 0, dev_bytes = 0;
    std::vector<double> x, v, f;     // input until admission, final state after it
    std::vector<mix_region> regions;
    int64_t steps_total = 0, steps_done = 0;
    unsigned char* dmem = nullptr;   // one allocation: x, v, f, workspace
    double t_submit = -1, t_admit = -1, t_done = -1;
};

}  // namespace

struct mix_server {
    mix_server_options opt{};
    cudaStream_t stream = nullptr;
    size_t budget = 0, in_use = 0;
    int64_t active_atoms = 0;
    int64_t next_id = 1;
    std::deque<int64_t> queue;
    std::vector<int64_t> active;
    std::map<int64_t, Request> req;
    mix_batch* batch = nullptr;
    bool dirty = true;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::chrono::steady_clock::time_point t0;
    std::string err;
};

namespace {

int sfail(mix_server* s, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s->err = buf;
    return code;
}

double now(const mix_server* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

size_t state_bytes(int64_t n) { return round256((size_t)(n > 0 ? n : 1) * 4 * sizeof(double)); }

// release a request's device memory and context (its host vectors stay)
void release(mix_server* s, Request& r) {
    if (r.ctx) {
        mix_destroy(r.ctx);
        r.ctx = nullptr;
    }
    if (r.dmem) {
        cudaFreeAsync(r.dmem, s->stream);
        r.dmem = nullptr;
        s->in_use -= r.dev_bytes;
        s->active_atoms -= r.n;
    }
}

void drop_batch(mix_server* s) {
    if (s->batch) mix_batch_destroy(s->batch);
    s->batch = nullptr;
    s->dirty = true;
}

// allocate, upload and bind one queued request; MIX_ENOMEM leaves it queued
int admit(mix_server* s, Request& r) {
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, r.dev_bytes, s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MIX_ENOMEM;
    }
    r.dmem = static_cast<unsigned char*>(p);
    s->in_use += r.dev_bytes;
    s->active_atoms += r.n;
    const size_t sb = state_bytes(r.n);
    double* dx = reinterpret_cast<double*>(r.dmem);
    double* dv = reinterpret_cast<double*>(r.dmem + sb);
    double* df = reinterpret_cast<double*>(r.dmem + 2 * sb);
    void* ws = r.dmem + 3 * sb;
    const size_t bytes = (size_t)r.n * 4 * sizeof(double);
    e = cudaMemsetAsync(df, 0, sb, s->stream);
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dx, r.x.data(), bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dv, r.v.data(), bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return sfail(s, MIX_ECUDA, "admission upload: %s", cudaGetErrorString(e));
    int st = mix_bind(r.ctx, dx, dv, df, ws);
    if (!st) st = mix_set_regions(r.ctx, r.regions.data(), (int)r.regions.size());
    if (!st) st = mix_forces(r.ctx);
    if (!st) st = mix_sync(r.ctx);
    return st;
}

void finish(mix_server* s, Request& r, int state, int status) {
    r.state = state;
    r.status = status;
    r.t_done = now(s);
    if (state == MIX_REQ_DONE && r.ctx) {
        int64_t step = 0;
        r.f.assign(r.x.size(), 0.0);
        const int st = mix_get_state(r.ctx, r.x.data(), r.v.data(), r.f.data(), &step);
        if (st) {
            r.state = MIX_REQ_FAILED;
            r.status = st;
        }
    }
    release(s, r);
}

}  // namespace

extern "C" {

int mix_admission_plan(const size_t* need, const int64_t* atoms, int n_queued, size_t bytes_free, int64_t atoms_free,
                       int active, int max_active, int fifo, int* admit) {
    if (n_queued < 0 || (n_queued > 0 && (!need || !atoms || !admit))) return MIX_EINVAL;
    int count = 0;
    for (int k = 0; k < n_queued; ++k) {
        admit[k] = 0;
        const bool slot = max_active <= 0 || active + count < max_active;
        const bool mem = need[k] <= bytes_free;
        // a request above the atom cap runs alone rather than never
        const bool cap = atoms_free < 0 || atoms[k] <= atoms_free || (active + count == 0);
        if (slot && mem && cap) {
            admit[k] = 1;
            ++count;
            bytes_free -= need[k];
            if (atoms_free >= 0) atoms_free = std::max<int64_t>(0, atoms_free - atoms[k]);
        } else if (fifo) {
            // the rest of the queue waits behind this request
            for (int j = k + 1; j < n_queued; ++j) admit[j] = 0;
            break;
        }
    }
    return count;
}

int mix_server_create(const mix_server_options* opt, void* cuda_stream, mix_server** out) {
    if (!out || !opt) return MIX_EINVAL;
    *out = nullptr;
    if (!(opt->dt_fs > 0) || opt->max_active < 0 || opt->max_active_atoms < 0) return MIX_EINVAL;
    mix_server* s = new (std::nothrow) mix_server();
    if (!s) return MIX_ENOMEM;
    s->opt = *opt;
    s->stream = (cudaStream_t)cuda_stream;
    s->t0 = std::chrono::steady_clock::now();
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        delete s;
        return MIX_ECUDA;
    }
    if (opt->hbm_budget > 0) {
        s->budget = opt->hbm_budget;
    } else {
        const size_t reserve = opt->hbm_reserve > 0 ? opt->hbm_reserve : ((size_t)2 << 30);
        s->budget = fr > reserve ? fr - reserve : 0;
    }
    if (s->budget == 0) {
        delete s;
        return MIX_ENOMEM;
    }
    if (cudaEventCreate(&s->e0) != cudaSuccess || cudaEventCreate(&s->e1) != cudaSuccess) {
        delete s;
        return MIX_ECUDA;
    }
    *out = s;
    return MIX_OK;
}

int mix_server_submit(mix_server* s, const mix_system* sys, const mix_ace* a, const mix_spline* sp,
                      const mix_options* opt, const mix_region* regions, int n_regions, const double* x_host,
                      const double* v_host, int64_t nsteps, int64_t* id) {
    if (!s) return MIX_EINVAL;
    if (!sys || !a || !sp || !opt || !id || nsteps < 0 || n_regions < 0 || (n_regions > 0 && !regions) ||
        (sys->n_atoms > 0 && (!x_host || !v_host)))
        return sfail(s, MIX_EINVAL, "mix_server_submit: arguments");
    Request r;
    int st = mix_init(sys, a, sp, opt, s->stream, &r.ctx);
    if (st) return sfail(s, st, "mix_init: %s", mix_strerror(st));
    st = mix_workspace_bytes(r.ctx, &r.ws_bytes);
    if (st) {
        mix_destroy(r.ctx);
        return sfail(s, st, "mix_workspace_bytes");
    }
    r.n = sys->n_atoms;
    r.dev_bytes = 3 * state_bytes(r.n) + round256(std::max<size_t>(r.ws_bytes, 256));
    if (r.dev_bytes > s->budget) {
        mix_destroy(r.ctx);
        return sfail(s, MIX_ENOMEM, "request needs %zu device bytes, budget %zu", r.dev_bytes, s->budget);
    }
    r.x.assign(x_host, x_host + (size_t)r.n * 4);
    r.v.assign(v_host, v_host + (size_t)r.n * 4);
    r.regions.assign(regions, regions + n_regions);
    r.steps_total = nsteps;
    r.id = s->next_id++;
    r.t_submit = now(s);
    *id = r.id;
    s->queue.push_back(r.id);
    s->req.emplace(r.id, std::move(r));
    return MIX_OK;
}

int mix_server_tick(mix_server* s, int max_steps, mix_tick_info* info) {
    if (!s) return MIX_EINVAL;
    if (max_steps < 1) return sfail(s, MIX_EINVAL, "max_steps >= 1");
    mix_tick_info ti;
    std::memset(&ti, 0, sizeof ti);
    auto ms_since = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
    };

    // 1. admission, in queue order
    const auto ta = std::chrono::steady_clock::now();
    if (!s->queue.empty()) {
        std::vector<size_t> need;
        std::vector<int64_t> atoms;
        for (int64_t q : s->queue) {
            need.push_back(s->req[q].dev_bytes);
            atoms.push_back(s->req[q].n);
        }
        std::vector<int> adm(need.size(), 0);
        const int64_t afree = s->opt.max_active_atoms > 0 ? std::max<int64_t>(0, s->opt.max_active_atoms - s->active_atoms)
                                                          : -1;
        mix_admission_plan(need.data(), atoms.data(), (int)need.size(), s->budget - s->in_use, afree,
                           (int)s->active.size(), s->opt.max_active, s->opt.fifo, adm.data());
        std::deque<int64_t> rest;
        bool out_of_memory = false;
        for (size_t k = 0; k < need.size(); ++k) {
            const int64_t q = s->queue[k];
            if (!adm[k] || out_of_memory) {
                rest.push_back(q);
                continue;
            }
            Request& r = s->req[q];
            const int st = admit(s, r);
            if (st == MIX_ENOMEM) {
                // the device had less free memory than the budget assumed
                out_of_memory = true;
                rest.push_back(q);
                continue;
            }
            if (st) {
                finish(s, r, MIX_REQ_FAILED, st);
                ++ti.failed;
                continue;
            }
            r.state = MIX_REQ_ACTIVE;
            r.t_admit = now(s);
            s->active.push_back(q);
            s->dirty = true;
            ++ti.admitted;
        }
        s->queue.swap(rest);
    }
    ti.admit_ms = ms_since(ta);

    // 2. requests that asked for no steps are done at once
    for (size_t k = 0; k < s->active.size();) {
        Request& r = s->req[s->active[k]];
        if (r.steps_done >= r.steps_total) {
            finish(s, r, MIX_REQ_DONE, MIX_OK);
            s->active.erase(s->active.begin() + k);
            s->dirty = true;
            ++ti.retired;
        } else {
            ++k;
        }
    }

    // 3. one batched graph over the active requests
    if (!s->active.empty()) {
        const auto tr = std::chrono::steady_clock::now();
        if (s->dirty) {
            if (s->batch) mix_batch_destroy(s->batch);
            s->batch = nullptr;
            std::vector<mix_ctx*> m;
            for (int64_t q : s->active) m.push_back(s->req[q].ctx);
            int st = mix_batch_create(m.data(), (int)m.size(), s->stream, &s->batch);
            if (st) return sfail(s, st, "mix_batch_create");
            // zero steps: builds the batch graph, so the timed steps below hold only GPU work
            st = mix_batch_step(s->batch, s->opt.dt_fs, 0);
            if (st) return sfail(s, st, "batch graph: %s", mix_batch_last_error(s->batch));
            s->dirty = false;
        }
        ti.rebuild_ms = ms_since(tr);
        int steps = max_steps;
        for (int64_t q : s->active) {
            const Request& r = s->req[q];
            steps = (int)std::min<int64_t>(steps, r.steps_total - r.steps_done);
        }
        ti.active_atoms = s->active_atoms;
        cudaEventRecord(s->e0, s->stream);
        int st = mix_batch_step(s->batch, s->opt.dt_fs, steps);
        cudaEventRecord(s->e1, s->stream);
        const cudaError_t e = cudaEventSynchronize(s->e1);
        if (e != cudaSuccess) return sfail(s, MIX_ECUDA, "tick: %s", cudaGetErrorString(e));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->e0, s->e1);
        ti.step_ms = steps > 0 ? ms / steps : 0.0;
        ti.steps = st ? 0 : steps;
        // 4. per-request status: failed requests leave, the rest advance
        for (size_t k = 0; k < s->active.size();) {
            Request& r = s->req[s->active[k]];
            const int rs = mix_sync(r.ctx);
            if (rs) {
                finish(s, r, MIX_REQ_FAILED, rs);
                s->active.erase(s->active.begin() + k);
                s->dirty = true;
                ++ti.failed;
                continue;
            }
            if (!st) r.steps_done += steps;
            if (r.steps_done >= r.steps_total) {
                finish(s, r, MIX_REQ_DONE, MIX_OK);
                s->active.erase(s->active.begin() + k);
                s->dirty = true;
                ++ti.retired;
                continue;
            }
            ++k;
        }
        if (st && ti.failed == 0) return sfail(s, st, "batch step: %s", mix_batch_last_error(s->batch));
    }
    if (s->dirty && s->batch) drop_batch(s);   // never keep a batch over destroyed members
    const cudaError_t e = cudaStreamSynchronize(s->stream);   // frees of retired requests
    if (e != cudaSuccess) return sfail(s, MIX_ECUDA, "tick: %s", cudaGetErrorString(e));
    ti.active = (int)s->active.size();
    ti.queued = (int)s->queue.size();
    ti.bytes_in_use = s->in_use;
    ti.t = now(s);
    if (info) *info = ti;
    return MIX_OK;
}

int mix_server_request(mix_server* s, int64_t id, mix_request_info* info) {
    if (!s || !info) return MIX_EINVAL;
    auto it = s->req.find(id);
    if (it == s->req.end()) return sfail(s, MIX_EINVAL, "unknown request %lld", (long long)id);
    const Request& r = it->second;
    info->state = r.state;
    info->status = r.status;
    info->n_atoms = r.n;
    info->steps_done = r.steps_done;
    info->steps_total = r.steps_total;
    info->device_bytes = r.dev_bytes;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    return MIX_OK;
}

int mix_server_fetch(mix_server* s, int64_t id, double* x_host, double* v_host, double* f_host) {
    if (!s) return MIX_EINVAL;
    auto it = s->req.find(id);
    if (it == s->req.end()) return sfail(s, MIX_EINVAL, "unknown request %lld", (long long)id);
    Request& r = it->second;
    if (r.state != MIX_REQ_DONE && r.state != MIX_REQ_FAILED) return sfail(s, MIX_ESTATE, "request not finished");
    const int status = r.status;
    if (r.state == MIX_REQ_DONE) {
        const size_t b = (size_t)r.n * 4 * sizeof(double);
        if (x_host && b) std::memcpy(x_host, r.x.data(), b);
        if (v_host && b) std::memcpy(v_host, r.v.data(), b);
        if (f_host && b) std::memcpy(f_host, r.f.data(), b);
    }
    s->req.erase(it);
    return status;
}

int mix_server_destroy(mix_server* s) {
    if (!s) return MIX_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->batch) mix_batch_destroy(s->batch);
    for (auto& kv : s->req) release(s, kv.second);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->e0) cudaEventDestroy(s->e0);
    if (s->e1) cudaEventDestroy(s->e1);
    delete s;
    return MIX_OK;
}

const char* mix_server_last_error(const mix_server* s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
