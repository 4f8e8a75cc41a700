// cwo_serve.cpp -- the native serving runtime declared in include/cwo_serve.h: per-size queues,
// slots (plan, stream, event, buffers), admission by a device-memory budget, mixed batches through
// cwo_propagate_items, and completion by event polling, all on the host thread that drives it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/cwo.h"
#include "../../include/cwo_serve.h"
#include "cwo_internal.h"

namespace {

cwo_status sfail(cwo_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    cwo::set_last_error(buf);
    return st;
}

cwo_status scuda(cudaError_t e, const char* what) {
    return sfail(CWO_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

using Clock = std::chrono::steady_clock;
double since(Clock::time_point t0) { return std::chrono::duration<double>(Clock::now() - t0).count(); }

constexpr int kMaxSlots = 8;

struct Slot {
    int n = 0, cap = 0;
    cwo_plan* plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    float2* inbuf = nullptr;                 // [cap][n][n] gathered inputs
    float2* outbuf = nullptr;                // [cap][n][n] outputs of a batch
    std::vector<long long> inflight;         // tickets of the batch on the GPU
    std::vector<cwo_item> items;             // host scratch of a launch
    size_t bytes = 0;                        // admission bytes of the batch in flight
};

struct Ticket {
    cwo_request req{};
    double t_done = -1.0;
};

bool pow2_side(int n) { return n >= CWO_MIN_SIDE && n <= CWO_MAX_SIDE && (n & (n - 1)) == 0; }

}  // namespace

struct cwo_server {
    int device = 0;
    std::vector<int> sizes;                      // ascending
    std::vector<std::vector<Slot>> slots;        // per size index
    std::vector<std::deque<long long>> queues;   // per size index
    std::vector<Ticket> tickets;
    size_t budget = 0, in_use = 0, peak = 0;
    long long batches = 0, completed = 0;
    Clock::time_point t0 = Clock::now();         // origin of the times cwo_server_done reports
    cudaEvent_t after = nullptr;

    int size_index(int n) const {
        for (size_t i = 0; i < sizes.size(); ++i)
            if (sizes[i] == n) return (int)i;
        return -1;
    }
};

namespace {

size_t batch_bytes(int n, int b) {
    size_t pb = 0;
    if (cwo_plan_device_bytes(n, n, b, &pb) != CWO_OK) return (size_t)-1;
    return pb + 2 * (size_t)b * (size_t)n * (size_t)n * 8u;
}

int admit_count(int queued, int capacity, size_t in_use, size_t budget, int n) {
    int b = std::min(queued, capacity);
    while (b > 0 && (batch_bytes(n, b) > budget || in_use > budget - batch_bytes(n, b))) b /= 2;
    return b;
}

cwo_status check_request(const cwo_server* srv, const cwo_request& r) {
    if (srv->size_index(r.n) < 0) return sfail(CWO_ERR_INVALID_ARG, "size %d is not served", r.n);
    if (r.type != CWO_ANGULAR && r.type != CWO_FRESNEL_CONV)
        return sfail(CWO_ERR_UNSUPPORTED, "request type %d: the server propagates CWO_ANGULAR and CWO_FRESNEL_CONV", r.type);
    if (!(r.wavelength > 0) || !std::isfinite(r.wavelength) || !(r.pitch > 0) || !std::isfinite(r.pitch) || !std::isfinite(r.z))
        return sfail(CWO_ERR_INVALID_ARG, "wavelength and pitch must be finite and > 0, z finite");
    if (r.type == CWO_FRESNEL_CONV && r.z == 0.0) return sfail(CWO_ERR_INVALID_ARG, "Fresnel diffraction needs z != 0");
    if (batch_bytes(r.n, 1) > srv->budget)
        return sfail(CWO_ERR_INVALID_ARG, "one %d^2 field needs more than the memory budget (%zu bytes)", r.n, srv->budget);
    const size_t fb = (size_t)r.n * (size_t)r.n * 8u;
    cwo_status st;
    if ((st = (cwo_status)cwo::check_device_buffer(r.field, fb, srv->device, "request field"))) return st;
    if (r.out && (st = (cwo_status)cwo::check_device_buffer(r.out, fb, srv->device, "request output"))) return st;
    return CWO_OK;
}

cwo_item item_of(const cwo_request& r) {
    cwo_item it{};
    it.z = r.z;
    it.lambda = r.wavelength;
    it.dx = r.pitch;
    it.dy = r.pitch;
    it.type = r.type;
    it.flags = 0;
    return it;
}

// Launch one batch of requests in slot s: a single request is propagated straight from its field
// to its output; a batch is gathered into the slot's input buffer, propagated into its output
// buffer and scattered to the requests' outputs.
cwo_status launch_batch(cwo_server* srv, Slot& s, const long long* tk_in, int b) {
    const long long field = (long long)s.n * s.n;
    // the batch's Fresnel requests after the others, so that cwo_propagate_items runs each route
    // (three passes; two separable line passes for Fresnel) as one sub-batch
    long long tk[cwo::kCopyMaxFields];
    int nt = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < b; ++i)
            if ((srv->tickets[tk_in[i]].req.type == CWO_FRESNEL_CONV) == (pass == 1)) tk[nt++] = tk_in[i];
    s.items.resize(b);
    for (int i = 0; i < b; ++i) s.items[i] = item_of(srv->tickets[tk[i]].req);
    cudaError_t e;
    cwo_status st;
    if (b == 1) {
        const cwo_request& r = srv->tickets[tk[0]].req;
        if ((st = cwo_propagate_items(s.plan, r.field, field, r.out ? r.out : (void*)s.outbuf, 1, s.items.data(), s.stream)))
            return st;
    } else {
        cwo::CopyList g{};
        bool scatter = false;
        for (int i = 0; i < b; ++i) {
            const cwo_request& r = srv->tickets[tk[i]].req;
            g.src[i] = (const float2*)r.field;
            g.dst[i] = s.inbuf + i * field;
            scatter = scatter || r.out;
        }
        if ((e = cwo::launch_copy_fields(g, b, field, s.stream)) != cudaSuccess) return scuda(e, "gather launch");
        if ((st = cwo_propagate_items(s.plan, s.inbuf, field, s.outbuf, b, s.items.data(), s.stream))) return st;
        if (scatter) {
            cwo::CopyList o{};
            for (int i = 0; i < b; ++i) {
                o.src[i] = s.outbuf + i * field;
                o.dst[i] = (float2*)srv->tickets[tk[i]].req.out;
            }
            if ((e = cwo::launch_copy_fields(o, b, field, s.stream)) != cudaSuccess) return scuda(e, "scatter launch");
        }
    }
    if ((e = cudaEventRecord(s.ev, s.stream)) != cudaSuccess) return scuda(e, "slot event record");
    s.inflight.assign(tk, tk + b);
    ++srv->batches;
    return CWO_OK;
}

cwo_status dispatch(cwo_server* srv) {
    for (size_t si = 0; si < srv->sizes.size(); ++si) {      // smallest size first
        std::deque<long long>& q = srv->queues[si];
        for (Slot& s : srv->slots[si]) {
            if (q.empty()) break;
            if (!s.inflight.empty()) continue;
            const int b = admit_count((int)std::min<size_t>(q.size(), 1 << 20), s.cap, srv->in_use, srv->budget, s.n);
            if (b == 0) break;                               // retried after completions free memory
            long long tk[cwo::kCopyMaxFields];
            for (int i = 0; i < b; ++i) {
                tk[i] = q.front();
                q.pop_front();
            }
            cwo_status st = launch_batch(srv, s, tk, b);
            if (st) {                                        // put the requests back, in order
                for (int i = b - 1; i >= 0; --i) q.push_front(tk[i]);
                return st;
            }
            s.bytes = batch_bytes(s.n, b);
            srv->in_use += s.bytes;
            srv->peak = std::max(srv->peak, srv->in_use);
        }
    }
    return CWO_OK;
}

// collect finished batches; `now` is the time stamped on their requests
cwo_status poll(cwo_server* srv, double now, int* done) {
    int d = 0;
    for (auto& v : srv->slots)
        for (Slot& s : v) {
            if (s.inflight.empty()) continue;
            const cudaError_t e = cudaEventQuery(s.ev);
            if (e == cudaErrorNotReady) {
                (void)cudaGetLastError();                    // not an error: clear the record
                continue;
            }
            if (e != cudaSuccess) return scuda(e, "slot event query");
            for (long long t : s.inflight) srv->tickets[t].t_done = now;
            d += (int)s.inflight.size();
            s.inflight.clear();
            srv->in_use -= s.bytes;
            s.bytes = 0;
        }
    srv->completed += d;
    if (done) *done = d;
    return CWO_OK;
}

void destroy_slots(cwo_server* srv) {
    for (auto& v : srv->slots)
        for (Slot& s : v) {
            if (s.stream) cudaStreamSynchronize(s.stream);
            cwo_plan_destroy(s.plan);
            if (s.ev) cudaEventDestroy(s.ev);
            if (s.stream) cudaStreamDestroy(s.stream);
            cudaFree(s.inbuf);
            cudaFree(s.outbuf);
        }
    srv->slots.clear();
}

}  // namespace

extern "C" {

cwo_status cwo_server_batch_bytes(int n, int b, size_t* bytes) {
    if (!bytes) return sfail(CWO_ERR_INVALID_ARG, "bytes is NULL");
    if (!pow2_side(n) || b < 1 || b > 65535) return sfail(CWO_ERR_INVALID_ARG, "n must be a power of two in [16, 4096], b in [1, 65535]");
    *bytes = batch_bytes(n, b);
    return CWO_OK;
}

cwo_status cwo_server_admit(int queued, int capacity, size_t in_use, size_t budget, int n, int* take) {
    if (!take) return sfail(CWO_ERR_INVALID_ARG, "take is NULL");
    if (queued < 0 || capacity < 1 || !pow2_side(n)) return sfail(CWO_ERR_INVALID_ARG, "bad admission arguments");
    *take = admit_count(queued, capacity, in_use, budget, n);
    return CWO_OK;
}

cwo_status cwo_server_create(int nsizes, const int* sizes, const int* max_batch, int slots_per_size,
                             size_t mem_budget, cwo_server** out) {
    if (!out) return sfail(CWO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nsizes < 1 || nsizes > 16 || !sizes || !max_batch) return sfail(CWO_ERR_INVALID_ARG, "1 to 16 sizes with their batch capacities");
    if (slots_per_size < 1 || slots_per_size > kMaxSlots) return sfail(CWO_ERR_INVALID_ARG, "slots_per_size must be in [1, %d]", kMaxSlots);
    std::vector<std::pair<int, int>> sz;
    for (int i = 0; i < nsizes; ++i) {
        if (!pow2_side(sizes[i])) return sfail(CWO_ERR_INVALID_ARG, "size %d: a power of two in [16, 4096]", sizes[i]);
        if (max_batch[i] < 1 || max_batch[i] > cwo::kCopyMaxFields)
            return sfail(CWO_ERR_INVALID_ARG, "size %d: batch capacity %d not in [1, %d]", sizes[i], max_batch[i], cwo::kCopyMaxFields);
        for (auto& p : sz)
            if (p.first == sizes[i]) return sfail(CWO_ERR_INVALID_ARG, "size %d given twice", sizes[i]);
        sz.emplace_back(sizes[i], max_batch[i]);
    }
    std::sort(sz.begin(), sz.end());
    cwo_server* srv = new (std::nothrow) cwo_server();
    if (!srv) return sfail(CWO_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&srv->device);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&srv->after, cudaEventDisableTiming);
    if (e != cudaSuccess) { delete srv; return scuda(e, "server set-up"); }
    size_t full = 0;
    srv->slots.resize(sz.size());
    srv->queues.resize(sz.size());
    for (size_t si = 0; si < sz.size(); ++si) {
        const int n = sz[si].first, cap = sz[si].second;
        srv->sizes.push_back(n);
        srv->slots[si].resize(slots_per_size);
        for (Slot& s : srv->slots[si]) {
            s.n = n;
            s.cap = cap;
            const size_t fb = (size_t)cap * n * n * sizeof(float2);
            cwo_status st = cwo_plan_create(n, n, CWO_DEFAULT_PITCH, CWO_DEFAULT_PITCH, CWO_DEFAULT_WAVELENGTH, 0.1,
                                            CWO_ANGULAR, 0, &s.plan);
            if (!st) st = cwo_plan_reserve(s.plan, cap);
            if (st) { destroy_slots(srv); cudaEventDestroy(srv->after); delete srv; return st; }
            // short requests on the higher-priority streams
            if ((e = cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, n <= 512 ? greatest : least)) ||
                (e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming)) || (e = cudaMalloc(&s.inbuf, fb)) ||
                (e = cudaMalloc(&s.outbuf, fb)) || (e = cudaMemset(s.inbuf, 0, fb)) || (e = cudaMemset(s.outbuf, 0, fb))) {
                cudaGetLastError();
                destroy_slots(srv);
                cudaEventDestroy(srv->after);
                delete srv;
                return e == cudaErrorMemoryAllocation ? sfail(CWO_ERR_OOM, "server buffers: out of device memory")
                                                      : scuda(e, "server slot set-up");
            }
            full += batch_bytes(n, cap);
        }
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { destroy_slots(srv); cudaEventDestroy(srv->after); delete srv; return scuda(e, "server set-up"); }
    srv->budget = mem_budget ? mem_budget : full;
    srv->t0 = Clock::now();
    *out = srv;
    return CWO_OK;
}

cwo_status cwo_server_destroy(cwo_server* srv) {
    if (!srv) return CWO_OK;
    destroy_slots(srv);
    if (srv->after) cudaEventDestroy(srv->after);
    delete srv;
    return CWO_OK;
}

cwo_status cwo_server_submit(cwo_server* srv, const cwo_request* req, long long* ticket) {
    if (!srv || !req || !ticket) return sfail(CWO_ERR_INVALID_ARG, "server, request and ticket are required");
    cwo_status st = check_request(srv, *req);
    if (st) return st;
    Ticket t;
    t.req = *req;
    srv->tickets.push_back(t);
    *ticket = (long long)srv->tickets.size() - 1;
    srv->queues[srv->size_index(req->n)].push_back(*ticket);
    return CWO_OK;
}

cwo_status cwo_server_after(cwo_server* srv, void* cuda_stream) {
    if (!srv) return sfail(CWO_ERR_INVALID_ARG, "server is NULL");
    cudaError_t e = cudaEventRecord(srv->after, (cudaStream_t)cuda_stream);
    for (auto& v : srv->slots)
        for (Slot& s : v)
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s.stream, srv->after, 0);
    return e == cudaSuccess ? CWO_OK : scuda(e, "ordering after the caller's stream");
}

cwo_status cwo_server_step(cwo_server* srv, int* completed) {
    if (!srv) return sfail(CWO_ERR_INVALID_ARG, "server is NULL");
    cwo_status st = dispatch(srv);
    if (st) return st;
    return poll(srv, since(srv->t0), completed);
}

int cwo_server_done(cwo_server* srv, long long ticket, double* t_done) {
    if (!srv || ticket < 0 || ticket >= (long long)srv->tickets.size()) return -1;
    const double t = srv->tickets[ticket].t_done;
    if (t < 0) return 0;
    if (t_done) *t_done = t;
    return 1;
}

cwo_status cwo_server_run(cwo_server* srv, const cwo_request* reqs, int nreq, double* t_done) {
    if (!srv || (nreq > 0 && (!reqs || !t_done)) || nreq < 0) return sfail(CWO_ERR_INVALID_ARG, "server, requests and t_done are required");
    for (int i = 0; i < nreq; ++i) {
        cwo_status st = check_request(srv, reqs[i]);
        if (st) return sfail(st, "request %d: %s", i, cwo_last_error());
    }
    std::vector<int> order(nreq);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].t_arrival < reqs[b].t_arrival; });
    const long long base = (long long)srv->tickets.size();
    srv->tickets.resize(base + nreq);
    for (int i = 0; i < nreq; ++i) srv->tickets[base + i].req = reqs[i];
    const Clock::time_point start = Clock::now();
    int next = 0, done = 0;
    while (done < nreq) {
        const double now = since(start);
        while (next < nreq && reqs[order[next]].t_arrival <= now) {
            const int k = order[next++];
            srv->queues[srv->size_index(reqs[k].n)].push_back(base + k);
        }
        cwo_status st = dispatch(srv);
        int d = 0;
        if (!st) st = poll(srv, since(start), &d);
        if (st) return st;
        done += d;
    }
    for (int i = 0; i < nreq; ++i) t_done[i] = srv->tickets[base + i].t_done;
    srv->tickets.resize(base);   // the run's own records: never handed out, all completed
    return CWO_OK;
}

cwo_status cwo_server_run_serial(cwo_server* srv, const cwo_request* reqs, int nreq, double* t_done) {
    if (!srv || (nreq > 0 && (!reqs || !t_done)) || nreq < 0) return sfail(CWO_ERR_INVALID_ARG, "server, requests and t_done are required");
    for (auto& v : srv->slots)
        for (Slot& s : v)
            if (!s.inflight.empty()) return sfail(CWO_ERR_INVALID_ARG, "the serial baseline needs an idle server");
    for (int i = 0; i < nreq; ++i) {
        cwo_status st = check_request(srv, reqs[i]);
        if (st) return sfail(st, "request %d: %s", i, cwo_last_error());
    }
    std::vector<int> order(nreq);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].t_arrival < reqs[b].t_arrival; });
    const Clock::time_point start = Clock::now();
    for (int k : order) {
        const cwo_request& r = reqs[k];
        while (since(start) < r.t_arrival) {
        }
        Slot& s = srv->slots[srv->size_index(r.n)][0];
        const cwo_item it = item_of(r);
        cwo_status st = cwo_propagate_items(s.plan, r.field, (long long)r.n * r.n, r.out ? r.out : (void*)s.outbuf, 1, &it, s.stream);
        if (st) return st;
        const cudaError_t e = cudaStreamSynchronize(s.stream);
        if (e != cudaSuccess) return scuda(e, "serial baseline");
        t_done[k] = since(start);
    }
    return CWO_OK;
}

cwo_status cwo_server_warm_up(cwo_server* srv) {
    if (!srv) return sfail(CWO_ERR_INVALID_ARG, "server is NULL");
    for (auto& v : srv->slots)
        for (Slot& s : v) {
            if (!s.inflight.empty()) return sfail(CWO_ERR_INVALID_ARG, "warm-up needs an idle server");
            const long long field = (long long)s.n * s.n;
            for (int b = 1; b <= std::min(2, s.cap); ++b)
                for (int type : {CWO_ANGULAR, CWO_FRESNEL_CONV}) {
                    std::vector<cwo_item> items(b);
                    for (auto& it : items) {
                        it = cwo_item{};
                        it.z = 0.1; it.lambda = 532e-9; it.dx = 8e-6; it.dy = 8e-6; it.type = type;
                    }
                    cudaError_t e = cudaSuccess;
                    cwo::CopyList g{};
                    for (int i = 0; i < b; ++i) {
                        g.src[i] = s.outbuf + i * field;     // exercises the gather and scatter copies
                        g.dst[i] = s.inbuf + i * field;
                    }
                    if (b > 1 && (e = cwo::launch_copy_fields(g, b, field, s.stream)) != cudaSuccess) return scuda(e, "warm-up copy");
                    cwo_status st = cwo_propagate_items(s.plan, s.inbuf, field, s.outbuf, b, items.data(), s.stream);
                    if (st) return st;
                    if ((e = cudaStreamSynchronize(s.stream)) != cudaSuccess) return scuda(e, "warm-up");
                }
            if (cudaMemsetAsync(s.inbuf, 0, (size_t)s.cap * field * sizeof(float2), s.stream) != cudaSuccess ||
                cudaStreamSynchronize(s.stream) != cudaSuccess)
                return scuda(cudaGetLastError(), "warm-up reset");
        }
    return CWO_OK;
}

cwo_status cwo_server_get_stats(const cwo_server* srv, cwo_server_stats* stats) {
    if (!srv || !stats) return sfail(CWO_ERR_INVALID_ARG, "server and stats are required");
    stats->batches = srv->batches;
    stats->completed = srv->completed;
    stats->mem_in_use = srv->in_use;
    stats->mem_peak = srv->peak;
    stats->mem_budget = srv->budget;
    return CWO_OK;
}

}  // extern "C"
