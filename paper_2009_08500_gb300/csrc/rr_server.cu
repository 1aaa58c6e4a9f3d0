// Continuous-batching evaluation server in the library (a worker thread).
//
// Requests (one fit's light curves for a batch of parameter vectors, host
// buffers, optionally with a cotangent for the adjoint) are queued by any
// host thread; the buffers must be page-locked memory mapped for the device,
// and their device addresses are looked up once, at submission.  The worker
// admits requests in arrival order whenever one of the server's streams is
// free and the request's device bytes (its workspace: the kernels read and
// write the host buffers in place) fit in the memory budget; it takes that
// memory from a stream-ordered pool on the request's stream (the pool keeps
// up to the budget, and reserves min(budget, 1 GiB) at creation), enqueues
// the request's kernels, records an event, and returns the memory on the
// same stream.  The choice of request and slot is made under the server's
// lock, the CUDA calls outside it.  After the request's kernels a one-thread
// kernel moves the context's device error word into a mapped word of the
// slot and clears it, so that a bounded device wait that gave up inside the
// request is reported as its RR_ETIMEOUT.  A host callback at the end of
// each request's stream work wakes the worker, which then reaps finished
// requests (event queries) and hands them to rr_server_poll.  Work of
// requests admitted at different times overlaps on the device; each request
// runs the same kernels as it would alone, so its results do not depend on
// the others.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rr_internal.h"

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    int64_t id = 0;
    rr_ctx* fit = nullptr;
    const double* times = nullptr;
    const int32_t* pb = nullptr;
    int32_t npt = 0;
    const double* params = nullptr;
    int32_t npv = 0;
    std::vector<int32_t> ss;
    std::vector<double> exptime;
    const void* grad_flux = nullptr;
    void* flux = nullptr;
    double* grad = nullptr;
    int32_t* status = nullptr;
    size_t bytes = 0;
    rr::InPlace in_place;      // the buffers' device addresses (all mapped page-locked memory)
    // t_arrival: the release time (not admitted before it), else the submit call
    int64_t t_arrival = 0, t_admit = 0, t_done = 0;
    int32_t result = RR_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t req = -1;          // request in flight, -1 = free
    int* err_word = nullptr;   // pinned: the fit's device error word after the request
};

}  // namespace

struct rr_server {
    int device = 0;
    size_t budget = 0, used = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;                       // waiting for admission, arrival order
    std::deque<int64_t> finished;                    // completed, not yet polled
    std::unordered_map<int64_t, Request> reqs;       // every request not yet released
    int64_t next_id = 0;
    bool stop = false;
    std::atomic<bool> woken{false};                  // a request's stream work has ended (callback)
    std::thread worker;
    std::string err;
};

namespace {

// Host callback enqueued after each request: wakes the worker.  It takes no
// lock and makes no CUDA call (the worker may hold the lock inside CUDA calls);
// a wake-up that comes between the worker's check and its wait is lost, and
// the worker's bounded wait (1 ms) covers it.
void CUDART_CB wake_worker(void* arg) {
    rr_server* s = static_cast<rr_server*>(arg);
    s->woken.store(true, std::memory_order_release);
    s->cv_work.notify_one();
}

// The fit's device error word after a request, into the slot's mapped host word, and cleared
// for the next request (a wait that gave up in another request of the same fit in flight at the
// same time is reported by whichever of them takes the word first).
__global__ void take_error_kernel(int* dev_word, int* host_word) { *host_word = atomicExch(dev_word, 0); }

// Enqueue one admitted request on its slot's stream (lock not held).
void enqueue(rr_server* s, Request& r, Slot& sl) {
    void* scratch = nullptr;
    const size_t bytes = r.bytes > 0 ? r.bytes : 256;
    cudaError_t e = cudaMallocFromPoolAsync(&scratch, bytes, s->pool, sl.stream);
    if (e == cudaSuccess) {
        r.result = r.in_place.ok
                       ? rr::run_in_place(r.fit, r.in_place, r.npt, r.npv, r.ss.data(), r.exptime.data(), scratch,
                                          bytes, sl.stream, false)
                       : rr_enqueue_host(r.fit, r.times, r.pb, r.npt, r.params, r.npv, r.ss.data(),
                                         r.exptime.data(), r.grad_flux, r.flux, r.grad, r.status, scratch, bytes,
                                         sl.stream);
        cudaFreeAsync(scratch, sl.stream);
        *sl.err_word = 0;
        if (r.result == RR_OK) {
            take_error_kernel<<<1, 1, 0, sl.stream>>>(r.fit->d_err, sl.err_word);
            if (cudaGetLastError() != cudaSuccess) r.result = RR_ECUDA;
        }
    } else {
        r.result = RR_ENOMEM;
    }
    if ((e = cudaEventRecord(sl.done, sl.stream)) != cudaSuccess && r.result == RR_OK) r.result = RR_ECUDA;
    cudaLaunchHostFunc(sl.stream, wake_worker, s);
}

// Admit and launch queued requests while a slot and memory are free.  The choice is made under
// the lock; the CUDA calls that enqueue a request run without it, so that submissions and polls
// do not wait for them (only this thread touches the slots, and an admitted request stays in
// `reqs` until it has been reported finished).
void admit(rr_server* s, std::unique_lock<std::mutex>& lk) {
    while (!s->queue.empty()) {
        Request& r = s->reqs[s->queue.front()];
        if (r.t_arrival > now_ns()) break;                // in order: not released yet
        if (s->used + r.bytes > s->budget) break;        // in order: wait for memory
        int slot = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (s->slots[i].req < 0) { slot = (int)i; break; }
        if (slot < 0) break;
        s->queue.pop_front();
        Slot& sl = s->slots[slot];
        r.t_admit = now_ns();
        s->used += r.bytes;
        sl.req = r.id;
        lk.unlock();
        enqueue(s, r, sl);
        lk.lock();
    }
}

// Hand over requests whose stream has passed them (lock held).
void reap(rr_server* s) {
    for (Slot& sl : s->slots) {
        if (sl.req < 0) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        Request& r = s->reqs[sl.req];
        if (q != cudaSuccess && r.result == RR_OK) r.result = RR_ECUDA;
        if (r.result == RR_OK && *sl.err_word != 0) r.result = RR_ETIMEOUT;
        r.t_done = now_ns();
        s->used -= r.bytes;
        s->finished.push_back(r.id);
        sl.req = -1;
        s->cv_done.notify_all();
    }
}

void run(rr_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        reap(s);
        admit(s, lk);
        bool busy = false;
        for (const Slot& sl : s->slots) busy = busy || sl.req >= 0;
        if (s->stop && !busy && s->queue.empty()) return;
        if (!busy && s->queue.empty()) {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        if (!busy) {
            // idle until the head of the queue is released (or a submission wakes the thread)
            const int64_t wait_ns = s->reqs[s->queue.front()].t_arrival - now_ns();
            if (wait_ns > 50000) {
                s->cv_work.wait_for(lk, std::chrono::nanoseconds(std::min<int64_t>(wait_ns - 20000, 20000000)));
                continue;
            }
        }
        // requests in flight: sleep until a request's callback (or at most 1 ms: the
        // release time of the next queued request may come first)
        s->cv_work.wait_for(lk, std::chrono::microseconds(1000),
                            [s] { return s->woken.load(std::memory_order_acquire) || s->stop; });
        s->woken.store(false, std::memory_order_relaxed);
    }
}

}  // namespace

extern "C" rr_status rr_server_create(int32_t device, int32_t slots, size_t mem_budget, rr_server** out) {
    if (!out) return RR_EINVAL;
    *out = nullptr;
    if (slots < 1 || slots > 64 || mem_budget == 0) return RR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return RR_ECUDA;
    rr_server* s = new (std::nothrow) rr_server();
    if (!s) return RR_ENOMEM;
    s->device = device;
    s->budget = mem_budget;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        // keep the pool's memory between requests (up to the budget)
        uint64_t keep = mem_budget;
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->slots.resize(slots);
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.err_word, sizeof(int), cudaHostAllocDefault);
    }
    if (e == cudaSuccess) {
        // reserve min(budget, 1 GiB) of pool memory now, so that the first requests do not wait
        // for the pool to grow (it keeps what it holds, up to the budget)
        void* p = nullptr;
        const size_t reserve = std::min<size_t>(mem_budget, (size_t)1 << 30);
        e = cudaMallocFromPoolAsync(&p, reserve, s->pool, s->slots[0].stream);
        if (e == cudaSuccess) e = cudaFreeAsync(p, s->slots[0].stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->slots[0].stream);
    }
    if (e != cudaSuccess) {
        for (Slot& sl : s->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.err_word) cudaFreeHost(sl.err_word);
        }
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return RR_ECUDA;
    }
    s->worker = std::thread(run, s);
    *out = s;
    return RR_OK;
}

extern "C" rr_status rr_server_destroy(rr_server* s) {
    if (!s) return RR_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (Slot& sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
        cudaFreeHost(sl.err_word);
    }
    cudaMemPoolDestroy(s->pool);
    delete s;
    return RR_OK;
}

extern "C" int64_t rr_server_now_ns(void) { return now_ns(); }

namespace {

// [p, p + bytes) in page-locked host memory mapped for the device (both ends):
// the kernels of a served request read and write its buffers in place.
bool page_locked(const void* p, size_t bytes) { return !p || bytes == 0 || rr::mapped_host(p, bytes) != nullptr; }

}  // namespace

extern "C" int64_t rr_server_submit_at(rr_server* s, rr_ctx* fit, const double* times, const int32_t* pb_index,
                                       int32_t npt, const double* params, int32_t npv, const int32_t* ss,
                                       const double* exptime, const void* grad_flux, void* flux,
                                       double* grad_params, int32_t* pv_status, int64_t release_ns) {
    if (!s || !fit || !ss || !exptime || npt < 0 || npv < 0 || (npv > 0 && !params) ||
        (npv > 0 && npt > 0 && (!times || !flux)) || (grad_flux && !grad_params) || release_ns < 0)
        return -RR_EINVAL;
    rr::InPlace in_place;
    if (npv > 0) {
        // the mapping is looked up for the fit's device, current on this thread for the check only
        // (cudaSetDevice also binds the device's context to a thread that has made no CUDA call
        // yet; without one, no device address is reported)
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(fit->cfg.device) != cudaSuccess) {
            cudaGetLastError();
            return -RR_ECUDA;
        }
        struct Restore {
            int d, now;
            ~Restore() {
                if (d != now) cudaSetDevice(d);
            }
        } restore{prev, fit->cfg.device};
        // a request with times runs in place; one without (validity words only) is staged
        in_place = rr::map_in_place(fit, times, pb_index, npt, params, npv, grad_flux, flux, grad_params, pv_status);
        if (npt > 0 ? !in_place.ok
                    : !page_locked(params, (size_t)npv * fit->nparam * 8) || !page_locked(pv_status, (size_t)npv * 4))
            return -RR_EPAGEABLE;
    }
    Request r;
    r.in_place = in_place;
    r.fit = fit;
    r.times = times;
    r.pb = pb_index;
    r.npt = npt;
    r.params = params;
    r.npv = npv;
    r.ss.assign(ss, ss + fit->cfg.npb);
    r.exptime.assign(exptime, exptime + fit->cfg.npb);
    r.grad_flux = grad_flux;
    r.flux = flux;
    r.grad = grad_params;
    r.status = pv_status;
    r.bytes = rr::request_bytes_in_place(fit, npv, npt, grad_flux != nullptr);
    if (r.bytes > s->budget) return -RR_ENOMEM;
    r.t_arrival = release_ns > 0 ? release_ns : now_ns();
    int64_t id;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return -RR_ESTATE;
        id = r.id = s->next_id++;
        s->reqs.emplace(id, std::move(r));
        s->queue.push_back(id);
    }
    s->cv_work.notify_one();
    return id;
}

extern "C" int64_t rr_server_submit(rr_server* s, rr_ctx* fit, const double* times, const int32_t* pb_index,
                                    int32_t npt, const double* params, int32_t npv, const int32_t* ss,
                                    const double* exptime, const void* grad_flux, void* flux, double* grad_params,
                                    int32_t* pv_status) {
    return rr_server_submit_at(s, fit, times, pb_index, npt, params, npv, ss, exptime, grad_flux, flux, grad_params,
                               pv_status, 0);
}

extern "C" int32_t rr_server_poll(rr_server* s, int64_t* ids, int32_t* status, int64_t* times_ns, int32_t max,
                                  int32_t timeout_us) {
    if (!s || !ids || max < 1) return -RR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->finished.empty() && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [s] { return !s->finished.empty(); });
    int32_t n = 0;
    while (n < max && !s->finished.empty()) {
        const int64_t id = s->finished.front();
        s->finished.pop_front();
        auto it = s->reqs.find(id);
        ids[n] = id;
        if (status) status[n] = it->second.result;
        if (times_ns) {
            times_ns[3 * n] = it->second.t_arrival;
            times_ns[3 * n + 1] = it->second.t_admit;
            times_ns[3 * n + 2] = it->second.t_done;
        }
        s->reqs.erase(it);
        ++n;
    }
    return n;
}

extern "C" int32_t rr_server_pending(rr_server* s) {
    if (!s) return -RR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    return (int32_t)(s->reqs.size() - s->finished.size());
}
