// Serving: continuous batching of slp_eval requests on resident plans.
//
// A server holds a set of plans (meshes resident on the device), a number of
// execution slots per plan (a CUDA stream plus a scratch set each) and a
// device arena for request buffers whose size is the HBM budget left after
// the slots.  Requests (plan, n states, host input, host output) are queued by
// slp_server_submit.  One scheduler thread, the only thread issuing CUDA
// work, repeatedly
//   1. retires finished requests (their completion event has fired): stamps
//      the latency, returns their arena blocks, frees the slot;
//   2. admits queued requests in arrival order, skipping a request whose plan
//      has no free slot or whose buffers do not fit the arena right now, so
//      requests for other meshes and smaller requests flow past it (a request
//      larger than the whole arena is rejected at submission);
//   3. for an admitted request, enqueues on the slot's stream: the copy of
//      the inputs, one evaluation per state, the copy of the outputs and a
//      completion event.
// Work of different slots overlaps on the device; the host never waits on a
// stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "slp_plan_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device block (host-side bookkeeping only).
class Arena {
public:
    void init(char *base, int64_t size) {
        base_ = base;
        size_ = size;
        free_.clear();
        if (size > 0) free_[0] = size;
        used_ = 0;
        peak_ = 0;
    }
    // returns offset or -1
    int64_t alloc(int64_t n) {
        n = (n + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const int64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                used_ += n;
                peak_ = std::max(peak_, used_);
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t n) {
        n = (n + 255) / 256 * 256;
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        // merge with the next block
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        // merge with the previous block
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *ptr(int64_t off) const { return base_ + off; }
    int64_t size() const { return size_; }
    int64_t used() const { return used_; }
    int64_t peak() const { return peak_; }

private:
    char *base_ = nullptr;
    int64_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<int64_t, int64_t> free_;
};

struct Request {
    int64_t id = 0;
    int plan = 0;
    int n_states = 0;
    const void *h_in = nullptr;
    void *h_out = nullptr;
    int state = 0;  // SLP_REQ_*
    int slot = -1;
    int64_t off_in = -1, off_out = -1, bytes_in = 0, bytes_out = 0;
    Clock::time_point t_submit, t_admit, t_done;
    slp_status result = SLP_OK;
    std::string error;  // failure text, reported by slp_server_wait
};

struct Slot {
    int plan = 0;
    slp::DevPlan view;
    SlpExec exec;  // near-field branch
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t request = -1;
};

}  // namespace

struct slp_server_s {
    int device = 0;
    int kind = SLP_INPUT_NODAL_MAG;
    std::vector<slp_plan_s *> plans;
    std::vector<int64_t> in_bytes_per_state, out_bytes_per_state;  // device stride per state (256-byte multiple)
    std::vector<int64_t> in_host_bytes, out_host_bytes;              // packed host bytes per state
    std::vector<Slot> slots;
    std::vector<void *> allocs;
    Arena arena;
    void *arena_base = nullptr;
    int64_t budget = 0, scratch_bytes = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;        // queued request ids, arrival order
    std::map<int64_t, Request> reqs;  // all requests not yet collected
    int64_t next_id = 1;
    bool stop = false;
    std::thread worker;

    // statistics
    std::vector<double> lat_ms, wait_ms;
    int64_t completed = 0, rejected = 0, cancelled = 0, targets_done = 0, max_inflight = 0;
    Clock::time_point t_first_submit, t_last_done;
    bool any_submit = false;
    std::string last_error;
};

namespace {

void finish_locked(slp_server_s &S, Request &r, int state, slp_status st) {
    r.state = state;
    r.result = st;
    r.t_done = Clock::now();
    if (state == SLP_REQ_DONE) {
        S.completed++;
        S.targets_done += (int64_t)r.n_states * S.plans[r.plan]->N;
        S.lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
        S.wait_ms.push_back(std::chrono::duration<double, std::milli>(r.t_admit - r.t_submit).count());
        S.t_last_done = r.t_done;
    }
    S.cv_done.notify_all();
}

// Enqueue the request's work on its slot's stream (scheduler thread only).
slp_status launch_request(slp_server_s &S, Request &r, Slot &sl) {
    slp_plan_s &p = *S.plans[r.plan];
    char *din = S.arena.ptr(r.off_in), *dout = S.arena.ptr(r.off_out);
    // host buffers are packed; on the device every state starts on a 256-byte boundary
    const int64_t ib = S.in_bytes_per_state[r.plan], ob = S.out_bytes_per_state[r.plan];
    const int64_t ihb = S.in_host_bytes[r.plan], ohb = S.out_host_bytes[r.plan];
    cudaError_t e = cudaMemcpy2DAsync(din, (size_t)ib, r.h_in, (size_t)ihb, (size_t)ihb, (size_t)r.n_states,
                                      cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) return slp_fail(SLP_ERR_CUDA, "request %lld: copy in: %s", (long long)r.id, cudaGetErrorString(e));
    // the request's states share passes over the near-field operator
    std::vector<const void *> ins(r.n_states);
    std::vector<void *> outs(r.n_states);
    for (int k = 0; k < r.n_states; ++k) {
        ins[k] = din + k * ib;
        outs[k] = dout + k * ob;
    }
    const slp_status st = slp_run_states(p, sl.view, S.kind, ins.data(), outs.data(), r.n_states, sl.stream, &sl.exec,
                                         nullptr);
    if (st != SLP_OK) return st;
    e = cudaMemcpy2DAsync(r.h_out, (size_t)ohb, dout, (size_t)ob, (size_t)ohb, (size_t)r.n_states,
                          cudaMemcpyDeviceToHost, sl.stream);
    if (e != cudaSuccess) return slp_fail(SLP_ERR_CUDA, "request %lld: copy out: %s", (long long)r.id, cudaGetErrorString(e));
    e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess) return slp_fail(SLP_ERR_CUDA, "event record: %s", cudaGetErrorString(e));
    return SLP_OK;
}

void scheduler(slp_server_s *Sp) {
    slp_server_s &S = *Sp;
    cudaSetDevice(S.device);
    std::unique_lock<std::mutex> lk(S.mu);
    while (true) {
        // 1. retire
        bool progress = false;
        int inflight = 0;
        for (Slot &sl : S.slots) {
            if (sl.request < 0) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                ++inflight;
                continue;
            }
            Request &r = S.reqs[sl.request];
            S.arena.release(r.off_in, r.bytes_in);
            S.arena.release(r.off_out, r.bytes_out);
            if (q == cudaSuccess)
                finish_locked(S, r, SLP_REQ_DONE, SLP_OK);
            else {
                r.error = std::string("device error: ") + cudaGetErrorString(q);
                cudaGetLastError();
                finish_locked(S, r, SLP_REQ_FAILED, SLP_ERR_CUDA);
            }
            sl.request = -1;
            progress = true;
        }
        // 2. admit in arrival order, skipping what cannot start now: reserve a
        //    slot and arena blocks under the lock, launch after releasing it
        std::vector<int64_t> admitted;
        for (auto it = S.queue.begin(); it != S.queue.end();) {
            Request &r = S.reqs[*it];
            int slot = -1;
            for (size_t k = 0; k < S.slots.size(); ++k)
                if (S.slots[k].plan == r.plan && S.slots[k].request < 0) {
                    slot = (int)k;
                    break;
                }
            if (slot < 0) {
                ++it;
                continue;
            }
            const int64_t oi = S.arena.alloc(r.bytes_in);
            if (oi < 0) {
                ++it;
                continue;
            }
            const int64_t oo = S.arena.alloc(r.bytes_out);
            if (oo < 0) {
                S.arena.release(oi, r.bytes_in);
                ++it;
                continue;
            }
            r.off_in = oi;
            r.off_out = oo;
            r.slot = slot;
            r.state = SLP_REQ_RUNNING;
            r.t_admit = Clock::now();
            S.slots[slot].request = r.id;
            admitted.push_back(r.id);
            ++inflight;
            it = S.queue.erase(it);
            progress = true;
        }
        if (!admitted.empty()) {
            // requests are never erased from the map, so the references stay valid
            std::vector<Request *> rs;
            for (int64_t id : admitted) rs.push_back(&S.reqs[id]);
            lk.unlock();
            std::vector<slp_status> res(rs.size());
            std::vector<std::string> msg(rs.size());
            for (size_t i = 0; i < rs.size(); ++i) {
                res[i] = launch_request(S, *rs[i], S.slots[rs[i]->slot]);
                if (res[i] != SLP_OK) {
                    msg[i] = slp_last_error();
                    cudaStreamSynchronize(S.slots[rs[i]->slot].stream);
                }
            }
            lk.lock();
            for (size_t i = 0; i < rs.size(); ++i) {
                if (res[i] == SLP_OK) continue;
                Request &r = *rs[i];
                S.arena.release(r.off_in, r.bytes_in);
                S.arena.release(r.off_out, r.bytes_out);
                S.slots[r.slot].request = -1;
                --inflight;
                r.error = msg[i];
                finish_locked(S, r, SLP_REQ_FAILED, res[i]);
            }
        }
        S.max_inflight = std::max<int64_t>(S.max_inflight, inflight);
        if (S.stop && S.queue.empty() && inflight == 0) break;
        if (!progress) {
            // nothing changed: sleep briefly while work is in flight, else until a submission
            if (inflight > 0)
                S.cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                S.cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

slp_status slp_server_default_opts(slp_server_opts *o) {
    if (!o) return slp_fail(SLP_ERR_INVALID_ARG, "opts is NULL");
    memset(o, 0, sizeof *o);
    o->slots_per_plan = 2;
    o->hbm_budget_bytes = (int64_t)8 << 30;
    return SLP_OK;
}

slp_status slp_server_create(int n_plans, const slp_plan_t *plans, int input_kind, const slp_server_opts *opts,
                             slp_server_t *out) {
    if (!out) return slp_fail(SLP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_plans < 1 || !plans) return slp_fail(SLP_ERR_INVALID_ARG, "no plans");
    if (input_kind < SLP_INPUT_SIGMA || input_kind > SLP_INPUT_ELEMENT)
        return slp_fail(SLP_ERR_INVALID_ARG, "unknown input kind %d", input_kind);
    slp_server_opts o;
    if (opts)
        o = *opts;
    else
        slp_server_default_opts(&o);
    if (o.slots_per_plan < 1 || o.slots_per_plan > 16) return slp_fail(SLP_ERR_INVALID_ARG, "slots_per_plan must be 1..16");
    const int dev = plans[0] ? plans[0]->device : -1;
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return slp_fail(SLP_ERR_INVALID_ARG, "plan %d is NULL", i);
        if (plans[i]->device < 0) return slp_fail(SLP_ERR_NO_DEVICE, "plan %d is host-only", i);
        if (plans[i]->device != dev) return slp_fail(SLP_ERR_INVALID_ARG, "all plans of a server must share a device");
        const slp_status ks = slp_check_kind(*plans[i], input_kind);
        if (ks != SLP_OK) return ks;
    }
    SlpDeviceGuard g(dev);
    slp_server_s *S = new slp_server_s();
    S->device = dev;
    S->kind = input_kind;
    S->budget = o.hbm_budget_bytes;
    auto cleanup = [&](slp_status st) {
        for (Slot &sl : S->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            slp_exec_destroy(sl.exec);
        }
        for (void *p : S->allocs) cudaFree(p);
        delete S;
        return st;
    };
    for (int i = 0; i < n_plans; ++i) {
        slp_plan_s &p = *plans[i];
        S->plans.push_back(plans[i]);
        const int64_t es = p.prec == 64 ? 8 : 4;
        const int64_t per_in = slp_input_count(p, input_kind);
        S->in_bytes_per_state.push_back(((es * per_in + 255) / 256) * 256);
        S->out_bytes_per_state.push_back(((es * p.N + 255) / 256) * 256);
        S->in_host_bytes.push_back(es * per_in);
        S->out_host_bytes.push_back(es * p.N);
        for (int k = 0; k < o.slots_per_plan; ++k) {
            Slot sl;
            sl.plan = i;
            if (k == 0) {
                sl.view = p.dp;
            } else {
                int64_t nb = 0;
                const slp_status st = slp_alloc_scratch(p, sl.view, S->allocs, &nb);
                if (st != SLP_OK) return cleanup(st);
                S->scratch_bytes += nb;
            }
            if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
                slp_exec_create(sl.exec) != cudaSuccess) {
                S->slots.push_back(sl);
                return cleanup(slp_fail(SLP_ERR_CUDA, "stream/event creation failed"));
            }
            S->slots.push_back(sl);
        }
    }
    const int64_t arena = S->budget - S->scratch_bytes;
    if (arena < (1 << 20))
        return cleanup(slp_fail(SLP_ERR_OOM, "HBM budget %lld bytes leaves no room for requests after %lld bytes of slots",
                                (long long)S->budget, (long long)S->scratch_bytes));
    if (cudaMalloc(&S->arena_base, (size_t)arena) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(slp_fail(SLP_ERR_OOM, "arena of %lld bytes", (long long)arena));
    }
    S->allocs.push_back(S->arena_base);
    S->arena.init((char *)S->arena_base, arena);
    S->worker = std::thread(scheduler, S);
    *out = S;
    return SLP_OK;
}

slp_status slp_server_submit(slp_server_t S, int plan_index, int n_states, const void *h_in, void *h_out,
                             int64_t *request_id) {
    if (!S || !h_in || !h_out || !request_id) return slp_fail(SLP_ERR_INVALID_ARG, "NULL argument");
    if (plan_index < 0 || plan_index >= (int)S->plans.size()) return slp_fail(SLP_ERR_INVALID_ARG, "bad plan index");
    if (n_states < 1) return slp_fail(SLP_ERR_INVALID_ARG, "n_states must be positive");
    Request r;
    r.plan = plan_index;
    r.n_states = n_states;
    r.h_in = h_in;
    r.h_out = h_out;
    r.bytes_in = (int64_t)n_states * S->in_bytes_per_state[plan_index];
    r.bytes_out = (int64_t)n_states * S->out_bytes_per_state[plan_index];
    r.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return slp_fail(SLP_ERR_INVALID_ARG, "server is shutting down");
    r.id = S->next_id++;
    *request_id = r.id;
    if (!S->any_submit) {
        S->any_submit = true;
        S->t_first_submit = r.t_submit;
    }
    if (r.bytes_in + r.bytes_out + 512 > S->arena.size()) {
        // can never be admitted under the budget
        r.state = SLP_REQ_REJECTED;
        r.result = SLP_ERR_OOM;
        r.t_done = r.t_submit;
        S->rejected++;
        S->reqs[r.id] = r;
        S->cv_done.notify_all();
        return SLP_OK;
    }
    r.state = SLP_REQ_QUEUED;
    S->reqs[r.id] = r;
    S->queue.push_back(r.id);
    S->cv_work.notify_all();
    return SLP_OK;
}

slp_status slp_server_status(slp_server_t S, int64_t request_id, int *state, slp_status *result) {
    if (!S || !state) return slp_fail(SLP_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return slp_fail(SLP_ERR_INVALID_ARG, "unknown request %lld", (long long)request_id);
    *state = it->second.state;
    if (result) *result = it->second.result;
    return SLP_OK;
}

slp_status slp_server_wait(slp_server_t S, int64_t request_id, double timeout_s, int *state) {
    if (!S) return slp_fail(SLP_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return slp_fail(SLP_ERR_INVALID_ARG, "unknown request %lld", (long long)request_id);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 3600.0);
    while (it->second.state == SLP_REQ_QUEUED || it->second.state == SLP_REQ_RUNNING) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            (it->second.state == SLP_REQ_QUEUED || it->second.state == SLP_REQ_RUNNING)) {
            if (state) *state = it->second.state;
            return slp_fail(SLP_ERR_TIMEOUT, "request %lld not finished after %.3f s", (long long)request_id, timeout_s);
        }
    }
    if (state) *state = it->second.state;
    if (it->second.result != SLP_OK)
        return slp_fail(it->second.result, "request %lld: %s", (long long)request_id,
                        it->second.error.empty() ? slp_status_string(it->second.result) : it->second.error.c_str());
    return SLP_OK;
}

slp_status slp_server_cancel(slp_server_t S, int64_t request_id) {
    if (!S) return slp_fail(SLP_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return slp_fail(SLP_ERR_INVALID_ARG, "unknown request %lld", (long long)request_id);
    if (it->second.state != SLP_REQ_QUEUED) return slp_fail(SLP_ERR_INVALID_ARG, "request is not queued");
    S->queue.erase(std::find(S->queue.begin(), S->queue.end(), request_id));
    it->second.state = SLP_REQ_CANCELLED;
    it->second.result = SLP_ERR_INVALID_ARG;
    it->second.t_done = Clock::now();
    S->cancelled++;
    S->cv_done.notify_all();
    return SLP_OK;
}

slp_status slp_server_stats(slp_server_t S, slp_server_statistics *st) {
    if (!S || !st) return slp_fail(SLP_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(st, 0, sizeof *st);
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->cancelled = S->cancelled;
    st->queued = (int64_t)S->queue.size();
    st->targets_done = S->targets_done;
    st->latency_p50_ms = percentile(S->lat_ms, 0.50);
    st->latency_p99_ms = percentile(S->lat_ms, 0.99);
    st->latency_max_ms = S->lat_ms.empty() ? 0.0 : *std::max_element(S->lat_ms.begin(), S->lat_ms.end());
    st->queue_wait_p50_ms = percentile(S->wait_ms, 0.50);
    st->queue_wait_p99_ms = percentile(S->wait_ms, 0.99);
    st->makespan_s = S->completed ? std::chrono::duration<double>(S->t_last_done - S->t_first_submit).count() : 0.0;
    st->arena_bytes = S->arena.size();
    st->arena_peak_bytes = S->arena.peak();
    st->slot_scratch_bytes = S->scratch_bytes;
    st->n_slots = (int64_t)S->slots.size();
    st->max_inflight = S->max_inflight;
    return SLP_OK;
}

slp_status slp_server_destroy(slp_server_t S) {
    if (!S) return SLP_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        // queued requests are cancelled; running ones finish
        for (int64_t id : S->queue) {
            Request &r = S->reqs[id];
            r.state = SLP_REQ_CANCELLED;
            r.result = SLP_ERR_INVALID_ARG;
            S->cancelled++;
        }
        S->queue.clear();
        S->stop = true;
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    SlpDeviceGuard g(S->device);
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        slp_exec_destroy(sl.exec);
    }
    for (void *p : S->allocs) cudaFree(p);
    delete S;
    return SLP_OK;
}

}  // extern "C"
