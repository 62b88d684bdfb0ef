// server.cu -- continuous-batching request loop over one GPU (ncf_server_*).
//
// Requests (one ACF or CCF each, any size, any options) are admitted while
// others are running, as long as the estimated device memory of everything
// admitted stays within the server's budget and a slot is free; otherwise the
// submit call returns NCF_EBUSY and the caller retries later.  Each slot owns
// a host worker thread, a CUDA stream and an ncf_ctx (workspace cached across
// requests), so admitted requests run concurrently and their kernels overlap
// on the device.  Every request runs exactly the kernels of ncf_corr on its
// own stream and its own memory: its result does not depend on what else is
// in flight (the integer rectangle accumulators are exact; the floating-point
// ones differ at most by summation order).
//
// Host buffers of a request (t, x, s, y, lags) must stay valid until
// ncf_server_wait has returned for its ticket.  Series that many requests
// share can be made resident (ncf_server_put): they are copied to the device
// once, charged to the budget, and requests name them by handle.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// A series held in device memory for the server's lifetime (or until dropped).
struct Resident {
    double *t = nullptr, *x = nullptr;
    int64_t n = 0;
    double t_first = 0.0, t_last = 0.0;  // host copies for the admission estimate
    size_t bytes = 0;
    int refs = 0;                         // admitted requests using it
};

struct Request {
    uint64_t ticket = 0;
    ncf_request req{};
    const Resident *rx = nullptr, *ry = nullptr;
    size_t est_bytes = 0;
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    ncf_status status = NCF_OK;
    std::string err;
    std::vector<double> c, b;
    std::vector<int64_t> count;
};

struct Slot {
    ncf_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    double *dbuf = nullptr;  // inputs and outputs of the current request
    size_t dcap = 0;
    std::thread th;
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device memory one request needs: the slot buffer of run_one (its own copies of
// the inputs, its lags and outputs) plus the context workspace of its ncf_corr
// call, sized by ncf_workspace_bytes from the request's sizes, time span and
// largest lag before anything is allocated; used for admission against the
// server's budget.  A request whose sizes the library refuses is charged its
// buffers only: ncf_corr then rejects it before allocating.
size_t estimate_bytes(const ncf_request &r, const Resident *rx, const Resident *ry) {
    const bool acf = r.s == nullptr && ry == nullptr;
    const int64_t nx = rx ? rx->n : r.nx, ny = acf ? 0 : (ry ? ry->n : r.ny), K = r.K;
    const int64_t cx = rx ? 0 : nx, cy = ry ? 0 : ny;  // points copied for this request
    const size_t own = align256(cx * 8) * 2 + align256(cy * 8) * 2 + align256(K * 8) * 4;
    double lo = rx ? rx->t_first : r.t[0], hi = rx ? rx->t_last : r.t[nx - 1];
    if (!acf) {
        lo = std::min(lo, ry ? ry->t_first : r.s[0]);
        hi = std::max(hi, ry ? ry->t_last : r.s[ny - 1]);
    }
    double max_tau = 0.0;
    for (int64_t k = 0; k < K; ++k) max_tau = std::max(max_tau, std::fabs(r.lags[k]));
    size_t ws = 0;
    if (ncf_workspace_bytes(nullptr, nx, ny, 1, K, hi - lo, max_tau, &r.opt, &ws, nullptr) != NCF_OK) ws = 0;
    return own + ws;
}

}  // namespace

struct ncf_server {
    int device = 0;
    size_t budget = 0, reserved = 0;
    std::vector<Slot> slots;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> requests;
    uint64_t next_ticket = 1;
    int busy = 0;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<double> latencies_ms;
    uint64_t completed = 0;
    std::map<uint64_t, Resident> resident;
    uint64_t next_series = 1;
};

namespace {

void run_one(ncf_server *srv, Slot &sl, Request &rq) {
    const ncf_request &r = rq.req;
    const bool acf = r.s == nullptr && rq.ry == nullptr;
    const int64_t nx = rq.rx ? rq.rx->n : r.nx, ny = acf ? 0 : (rq.ry ? rq.ry->n : r.ny), K = r.K;
    const int64_t cx = rq.rx ? 0 : nx, cy = rq.ry ? 0 : ny;  // points copied for this request
    const size_t need = align256(cx * 8) * 2 + align256(cy * 8) * 2 + align256(K * 8) + align256(K * 8) * 2 +
                        align256(K * 8);
    if (need > sl.dcap) {
        if (sl.dbuf) cudaFree(sl.dbuf);
        sl.dbuf = nullptr;
        sl.dcap = 0;
        if (cudaMalloc(&sl.dbuf, need) != cudaSuccess) {
            cudaGetLastError();
            rq.status = NCF_ENOMEM;
            rq.err = "cudaMalloc of the request buffers failed";
            return;
        }
        sl.dcap = need;
    }
    char *p = reinterpret_cast<char *>(sl.dbuf);
    auto take = [&](size_t bytes) { char *q = p; p += align256(bytes); return reinterpret_cast<double *>(q); };
    double *dt, *dx, *ds = nullptr, *dy = nullptr;
    if (rq.rx) {
        dt = rq.rx->t;
        dx = rq.rx->x;
    } else {
        dt = take(nx * 8);
        dx = take(nx * 8);
        cudaMemcpyAsync(dt, r.t, nx * 8, cudaMemcpyHostToDevice, sl.st);
        cudaMemcpyAsync(dx, r.x, nx * 8, cudaMemcpyHostToDevice, sl.st);
    }
    if (!acf) {
        if (rq.ry) {
            ds = rq.ry->t;
            dy = rq.ry->x;
        } else {
            ds = take(ny * 8);
            dy = take(ny * 8);
            cudaMemcpyAsync(ds, r.s, ny * 8, cudaMemcpyHostToDevice, sl.st);
            cudaMemcpyAsync(dy, r.y, ny * 8, cudaMemcpyHostToDevice, sl.st);
        }
    }
    double *dl = take(K * 8), *dc = take(K * 8), *db = take(K * 8);
    int64_t *dn = reinterpret_cast<int64_t *>(take(K * 8));
    cudaMemcpyAsync(dl, r.lags, K * 8, cudaMemcpyHostToDevice, sl.st);
    rq.status = ncf_corr(sl.ctx, dt, dx, nx, ds, dy, ny, dl, K, &r.opt, dc, db, dn, sl.st);
    if (rq.status != NCF_OK) {
        rq.err = ncf_last_error(sl.ctx);
        cudaStreamSynchronize(sl.st);
        return;
    }
    rq.c.resize(K);
    rq.b.resize(K);
    rq.count.resize(K);
    cudaMemcpyAsync(rq.c.data(), dc, K * 8, cudaMemcpyDeviceToHost, sl.st);
    cudaMemcpyAsync(rq.b.data(), db, K * 8, cudaMemcpyDeviceToHost, sl.st);
    cudaMemcpyAsync(rq.count.data(), dn, K * 8, cudaMemcpyDeviceToHost, sl.st);
    if (cudaStreamSynchronize(sl.st) != cudaSuccess) {
        rq.status = NCF_ECUDA;
        rq.err = cudaGetErrorString(cudaGetLastError());
    }
    (void)srv;
}

void worker(ncf_server *srv, int idx) {
    Slot &sl = srv->slots[idx];
    cudaSetDevice(srv->device);
    for (;;) {
        std::shared_ptr<Request> rq;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->stop || !srv->queue.empty(); });
            if (srv->stop && srv->queue.empty()) return;
            rq = srv->queue.front();
            srv->queue.pop_front();
            ++srv->busy;
        }
        rq->t_start = Clock::now();
        run_one(srv, sl, *rq);
        rq->t_done = Clock::now();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            rq->done = true;
            --srv->busy;
            srv->latencies_ms.push_back(
                std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count());
            ++srv->completed;
        }
        srv->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

ncf_status ncf_server_create(int device, size_t mem_budget_bytes, int slots, ncf_server **out) {
    if (!out || slots < 1 || slots > 64) return NCF_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return NCF_ECUDA;
    }
    auto *srv = new ncf_server();
    srv->device = device;
    srv->budget = mem_budget_bytes;
    srv->slots.resize(slots);
    for (auto &sl : srv->slots) {
        if (ncf_create(&sl.ctx, device) != NCF_OK ||
            cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto &s2 : srv->slots) {
                if (s2.ctx) ncf_destroy(s2.ctx);
                if (s2.st) cudaStreamDestroy(s2.st);
            }
            delete srv;
            return NCF_ECUDA;
        }
    }
    for (int i = 0; i < slots; ++i) srv->slots[i].th = std::thread(worker, srv, i);
    *out = srv;
    return NCF_OK;
}

ncf_status ncf_server_put(ncf_server *srv, const double *t, const double *x, int64_t n, uint64_t *series) {
    if (!srv || !t || !x || n < 2 || !series) return NCF_EINVAL;
    const size_t bytes = align256((size_t)n * 8) * 2;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->reserved + bytes > srv->budget) return NCF_EBUSY;
        srv->reserved += bytes;  // held while copying
    }
    Resident r;
    r.n = n;
    r.t_first = t[0];
    r.t_last = t[n - 1];
    r.bytes = bytes;
    char *mem = nullptr;
    cudaSetDevice(srv->device);
    if (cudaMalloc(&mem, bytes) != cudaSuccess ||
        cudaMemcpy(mem, t, (size_t)n * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(mem + align256((size_t)n * 8), x, (size_t)n * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        if (mem) cudaFree(mem);
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->reserved -= bytes;
        return NCF_ENOMEM;
    }
    r.t = reinterpret_cast<double *>(mem);
    r.x = reinterpret_cast<double *>(mem + align256((size_t)n * 8));
    std::lock_guard<std::mutex> lk(srv->mu);
    *series = srv->next_series++;
    srv->resident[*series] = r;
    return NCF_OK;
}

ncf_status ncf_server_drop(ncf_server *srv, uint64_t series) {
    if (!srv) return NCF_EINVAL;
    double *mem = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->resident.find(series);
        if (it == srv->resident.end()) return NCF_EINVAL;
        if (it->second.refs > 0) return NCF_EBUSY;
        mem = it->second.t;
        srv->reserved -= it->second.bytes;
        srv->resident.erase(it);
    }
    cudaSetDevice(srv->device);
    cudaFree(mem);
    return NCF_OK;
}

ncf_status ncf_server_submit(ncf_server *srv, const ncf_request *req, uint64_t *ticket) {
    if (!srv || !req || !ticket || !req->lags || req->K < 1) return NCF_EINVAL;
    if (!req->x_series && (!req->t || !req->x || req->nx < 2)) return NCF_EINVAL;
    if (!req->y_series && ((req->s == nullptr) != (req->y == nullptr) || (req->s && req->ny < 2)))
        return NCF_EINVAL;
    auto rq = std::make_shared<Request>();
    rq->req = *req;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (req->x_series) {
        auto it = srv->resident.find(req->x_series);
        if (it == srv->resident.end()) return NCF_EINVAL;
        rq->rx = &it->second;
    }
    if (req->y_series) {
        auto it = srv->resident.find(req->y_series);
        if (it == srv->resident.end()) return NCF_EINVAL;
        rq->ry = &it->second;
    }
    rq->est_bytes = estimate_bytes(*req, rq->rx, rq->ry);
    const int in_flight = (int)srv->queue.size() + srv->busy;
    if (in_flight >= (int)srv->slots.size() || srv->reserved + rq->est_bytes > srv->budget) return NCF_EBUSY;
    srv->reserved += rq->est_bytes;
    if (req->x_series) ++srv->resident[req->x_series].refs;
    if (req->y_series) ++srv->resident[req->y_series].refs;
    rq->ticket = srv->next_ticket++;
    rq->t_submit = Clock::now();
    srv->requests[rq->ticket] = rq;
    srv->queue.push_back(rq);
    *ticket = rq->ticket;
    srv->cv_work.notify_one();
    return NCF_OK;
}

ncf_status ncf_server_poll(ncf_server *srv, uint64_t ticket, int *done) {
    if (!srv || !done) return NCF_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->requests.find(ticket);
    if (it == srv->requests.end()) return NCF_EINVAL;
    *done = it->second->done ? 1 : 0;
    return NCF_OK;
}

ncf_status ncf_server_wait(ncf_server *srv, uint64_t ticket, double *c_out, double *b_out, int64_t *count_out,
                           double *latency_ms) {
    if (!srv) return NCF_EINVAL;
    std::shared_ptr<Request> rq;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->requests.find(ticket);
        if (it == srv->requests.end()) return NCF_EINVAL;
        rq = it->second;
        srv->cv_done.wait(lk, [&] { return rq->done; });
        srv->requests.erase(it);
        srv->reserved -= rq->est_bytes;
        if (rq->req.x_series) --srv->resident[rq->req.x_series].refs;
        if (rq->req.y_series) --srv->resident[rq->req.y_series].refs;
    }
    if (rq->status != NCF_OK) return rq->status;
    const size_t K = (size_t)rq->req.K;
    if (c_out) std::memcpy(c_out, rq->c.data(), K * 8);
    if (b_out) std::memcpy(b_out, rq->b.data(), K * 8);
    if (count_out) std::memcpy(count_out, rq->count.data(), K * 8);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count();
    return NCF_OK;
}

ncf_status ncf_server_latency(ncf_server *srv, double *p50_ms, double *p99_ms, uint64_t *completed) {
    if (!srv) return NCF_EINVAL;
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        v = srv->latencies_ms;
        if (completed) *completed = srv->completed;
    }
    if (v.empty()) {
        if (p50_ms) *p50_ms = 0.0;
        if (p99_ms) *p99_ms = 0.0;
        return NCF_OK;
    }
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
    if (p50_ms) *p50_ms = q(0.50);
    if (p99_ms) *p99_ms = q(0.99);
    return NCF_OK;
}

void ncf_server_destroy(ncf_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &sl : srv->slots)
        if (sl.th.joinable()) sl.th.join();
    cudaSetDevice(srv->device);
    for (auto &sl : srv->slots) {
        if (sl.dbuf) cudaFree(sl.dbuf);
        if (sl.ctx) ncf_destroy(sl.ctx);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    for (auto &kv : srv->resident) cudaFree(kv.second.t);
    delete srv;
}

}  // extern "C"
