// Request loop for serving prebuilt media (continuous batching over the
// boundary-to-coefficient maps).  Requests queue per medium on submit; worker
// threads, each with its own stream, pinned staging buffer and map workspace,
// admit the oldest queued requests of one medium into a batch while slots and
// device memory allow, run the batch (host-to-device copy of phi, map solve),
// and mark its requests done when the host sees the stream complete.  Results
// stay on the device until fetched or released; the device memory a request
// holds (its phi and u) is charged to the budget from admission to release.
// Every wait of a worker is a bounded condition-variable wait, rechecked in a
// loop, so destroy always ends the threads.
#include "internal.h"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace msp {

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct BatchMem {           // device buffer of one batch's results, shared by its requests
    double* u = nullptr;
    int refs = 0;
};

struct Request {
    int medium = 0;
    std::vector<double> phi;
    double t_submit = 0.0, t_done = 0.0;
    int state = 0;          // 0 queued, 1 admitted, 2 done, -1 failed
    msp_status status = MSP_OK;
    BatchMem* mem = nullptr;
    double* u = nullptr;    // this request's slice of mem->u
    long long bytes = 0;    // charged to the budget
};

struct Worker {
    std::thread th;
    cudaStream_t stream = nullptr;
    double* phi_dev = nullptr;
    double* pinned = nullptr;
    size_t pinned_n = 0, phi_n = 0;
    std::vector<MapWork> work;   // per medium
};

}  // namespace

struct Server {
    std::vector<Basis*> media;
    long long budget = 0;
    int max_slots = 0, max_batch = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::deque<uint64_t>> queues;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    long long mem_in_use = 0, mem_peak = 0;
    int slots_used = 0;
    bool stop = false;
    msp_server_stats st{};
    std::vector<Worker*> workers;
    Worker manual;   // n_workers == 0
    cudaStream_t free_stream = nullptr;   // stream-ordered frees of released results (no device-wide sync)
    // engine of the batch solves (read under the lock when a batch is admitted):
    // the map GEMM, or the plain FP64 iteration of msp_online_solve
    int engine = MSP_SERVE_MAP;
    double it_tol = 1e-8;
    int it_max_iter = 1000;
    std::vector<std::unique_ptr<std::mutex>> medium_mu;   // the iteration uses the basis's own workspace

    long long request_bytes(int m) const {
        const long long N = media[m]->N;
        return (long long)sizeof(double) * ((N + 1) * (N + 1) + 4 * N);
    }
};

namespace {

// Under the lock: pick the medium whose queue head is oldest and admit up to
// max_batch of its requests within the slot and memory limits.
bool admit(Server& S, int& medium, std::vector<uint64_t>& ids) {
    ids.clear();
    medium = -1;
    double oldest = 0.0;
    for (size_t m = 0; m < S.queues.size(); ++m) {
        if (S.queues[m].empty()) continue;
        const double t = S.reqs[S.queues[m].front()].t_submit;
        if (medium < 0 || t < oldest) {
            medium = (int)m;
            oldest = t;
        }
    }
    if (medium < 0) return false;
    const long long rb = S.request_bytes(medium);
    auto& q = S.queues[medium];
    while (!q.empty() && (int)ids.size() < S.max_batch && S.slots_used < S.max_slots &&
           S.mem_in_use + rb <= S.budget) {
        const uint64_t id = q.front();
        q.pop_front();
        Request& r = S.reqs[id];
        r.state = 1;
        r.bytes = rb;
        S.slots_used += 1;
        S.mem_in_use += rb;
        S.mem_peak = std::max(S.mem_peak, S.mem_in_use);
        ids.push_back(id);
    }
    return !ids.empty();
}

msp_status ensure_worker_buffers(Server& S, Worker& W, int medium, int B) {
    const Basis& Bs = *S.media[medium];
    const size_t n4 = 4 * (size_t)Bs.N;
    if (W.pinned_n < n4 * B) {
        if (W.pinned) cudaFreeHost(W.pinned);
        W.pinned = nullptr;
        W.pinned_n = 0;
        MSP_CUDA(cudaMallocHost((void**)&W.pinned, sizeof(double) * n4 * S.max_batch));
        W.pinned_n = n4 * S.max_batch;
    }
    if (W.phi_n < n4 * B) {
        if (W.phi_dev) cudaFree(W.phi_dev);
        W.phi_dev = nullptr;
        W.phi_n = 0;
        MSP_CUDA(cudaMalloc((void**)&W.phi_dev, sizeof(double) * n4 * S.max_batch));
        W.phi_n = n4 * S.max_batch;
    }
    if (W.work.size() < S.media.size()) W.work.resize(S.media.size());
    if (Bs.map_built && W.work[medium].cap < B) {
        map_work_free(W.work[medium]);
        MSP_TRY(map_work_alloc(Bs, S.max_batch, W.work[medium]));
    }
    return MSP_OK;
}

// The plain FP64 path for one batch: the CGLS iteration of msp_online_solve with
// the FP64 factor applied in FP64.  The iteration works in the basis's own
// buffers, so the batches of one medium take its lock.
msp_status iterative_batch(Server& S, int medium, const double* phi, int B, double* u, double tol, int max_iter,
                           cudaStream_t stream) {
    Basis& Bs = *S.media[medium];
    std::lock_guard<std::mutex> lk(*S.medium_mu[medium]);
    const int mode = Bs.bt_apply_mode;
    Bs.bt_apply_mode = 1;
    msp_status st = online_solve(Bs, phi, B, tol, max_iter, u, nullptr, nullptr, stream);
    Bs.bt_apply_mode = mode;
    // the reconstruction is still queued on this stream and reads the basis's
    // buffers: it must finish before another worker's batch may use them
    const cudaError_t e = cudaStreamSynchronize(stream);
    if (st == MSP_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    return st;
}

// Runs one admitted batch on the worker's stream and retires it.  Called without the lock.
msp_status run_batch(Server& S, Worker& W, cudaStream_t stream, int medium, const std::vector<uint64_t>& ids, int engine,
                     double it_tol, int it_max_iter) {
    const Basis& Bs = *S.media[medium];
    const int B = (int)ids.size();
    const size_t n4 = 4 * (size_t)Bs.N;
    const long long nn = (long long)(Bs.N + 1) * (Bs.N + 1);
    msp_status st = ensure_worker_buffers(S, W, medium, B);
    BatchMem* mem = nullptr;
    if (st == MSP_OK) {
        {
            std::lock_guard<std::mutex> lk(S.mu);
            for (int b = 0; b < B; ++b) {
                const Request& r = S.reqs[ids[b]];
                std::copy(r.phi.begin(), r.phi.end(), W.pinned + (size_t)b * n4);
            }
        }
        mem = new BatchMem();
        cudaError_t e = cudaMallocAsync((void**)&mem->u, sizeof(double) * nn * B, stream);
        if (e != cudaSuccess) {
            set_error(std::string("server: result buffer: ") + cudaGetErrorString(e));
            st = MSP_ERR_OOM;
        }
    }
    if (st == MSP_OK) {
        cudaError_t e = cudaMemcpyAsync(W.phi_dev, W.pinned, sizeof(double) * n4 * B, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) {
            set_error(std::string("server: phi copy: ") + cudaGetErrorString(e));
            st = MSP_ERR_CUDA;
        }
    }
    if (st == MSP_OK) {
        if (engine == MSP_SERVE_ITERATIVE_FP64) {
            st = iterative_batch(S, medium, W.phi_dev, B, mem->u, it_tol, it_max_iter, stream);
        } else if (!Bs.map_built) {
            set_error("server: the map engine needs msp_basis_build_map on every medium");
            st = MSP_ERR_STATE;
        } else {
            st = online_solve_map(Bs, W.phi_dev, B, mem->u, stream, &W.work[medium]);
        }
    }
    if (st == MSP_OK) {
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            set_error(std::string("server: batch: ") + cudaGetErrorString(e));
            st = MSP_ERR_CUDA;
        }
    }
    if (st == MSP_OK && engine == MSP_SERVE_MAP) st = map_work_check(W.work[medium], stream);
    const double t = now_ms();
    std::lock_guard<std::mutex> lk(S.mu);
    S.st.batches += 1;
    S.st.max_batch_seen = std::max(S.st.max_batch_seen, B);
    if (st == MSP_OK) {
        mem->refs = B;
        for (int b = 0; b < B; ++b) {
            Request& r = S.reqs[ids[b]];
            r.state = 2;
            r.t_done = t;
            r.mem = mem;
            r.u = mem->u + (long long)b * nn;
            // phi is no longer held on the device: charge only u from here
            const long long keep = (long long)sizeof(double) * nn;
            S.mem_in_use -= (r.bytes - keep);
            r.bytes = keep;
            r.phi.clear();
            r.phi.shrink_to_fit();
        }
        S.st.completed += B;
    } else {
        if (mem) {
            if (mem->u) cudaFreeAsync(mem->u, stream);
            delete mem;
        }
        for (int b = 0; b < B; ++b) {
            Request& r = S.reqs[ids[b]];
            r.state = -1;
            r.status = st;
            r.t_done = t;
            S.mem_in_use -= r.bytes;
            r.bytes = 0;
        }
        S.st.failed += B;
    }
    S.cv.notify_all();
    return st;
}

void worker_loop(Server* S, Worker* W) {
    cudaSetDevice(S->device);
    std::vector<uint64_t> ids;
    for (;;) {
        int medium = -1, engine = MSP_SERVE_MAP, it_max = 0;
        double it_tol = 0.0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (!S->stop && !admit(*S, medium, ids)) S->cv.wait_for(lk, std::chrono::milliseconds(2));
            engine = S->engine;
            it_tol = S->it_tol;
            it_max = S->it_max_iter;
            if (S->stop) {
                // give back anything admitted in the same pass
                for (uint64_t id : ids) {
                    Request& r = S->reqs[id];
                    r.state = -1;
                    r.status = MSP_ERR_INVALID_ARG;
                    S->mem_in_use -= r.bytes;
                    r.bytes = 0;
                }
                return;
            }
        }
        run_batch(*S, *W, W->stream, medium, ids, engine, it_tol, it_max);
    }
}

void release_locked(Server& S, std::unordered_map<uint64_t, Request>::iterator it) {
    Request& r = it->second;
    if (r.mem) {
        if (--r.mem->refs == 0) {
            cudaFreeAsync(r.mem->u, S.free_stream);
            delete r.mem;
        }
        r.mem = nullptr;
    }
    S.mem_in_use -= r.bytes;
    S.slots_used -= 1;
    S.st.released += 1;
    S.reqs.erase(it);
    S.cv.notify_all();
}

void free_worker(Worker& W) {
    for (auto& w : W.work) map_work_free(w);
    W.work.clear();
    if (W.phi_dev) cudaFree(W.phi_dev);
    if (W.pinned) cudaFreeHost(W.pinned);
    if (W.stream) cudaStreamDestroy(W.stream);
    W.phi_dev = nullptr;
    W.pinned = nullptr;
    W.stream = nullptr;
}

}  // namespace

}  // namespace msp

struct msp_server_s {
    msp::Server S;
};

using namespace msp;

extern "C" msp_status msp_server_create(const msp_basis* media, int n_media, long long mem_budget_bytes, int max_slots,
                                        int max_batch, int n_workers, msp_server* out) {
    clear_error();
    MSP_CHECK_ARG(media && out && n_media >= 1, "msp_server_create: need at least one medium");
    MSP_CHECK_ARG(mem_budget_bytes > 0 && max_slots >= 1, "msp_server_create: budget and slots must be positive");
    MSP_CHECK_ARG(max_batch >= 1 && max_batch <= 64, "msp_server_create: max_batch must lie in [1, 64]");
    MSP_CHECK_ARG(n_workers >= 0 && n_workers <= 16, "msp_server_create: n_workers must lie in [0, 16]");
    for (int m = 0; m < n_media; ++m) MSP_CHECK_ARG(media[m], "msp_server_create: NULL basis");
    auto* h = new msp_server_s();
    Server& S = h->S;
    for (int m = 0; m < n_media; ++m) {
        S.media.push_back(&media[m]->B);
        S.medium_mu.emplace_back(new std::mutex());
    }
    S.budget = mem_budget_bytes;
    S.max_slots = max_slots;
    S.max_batch = max_batch;
    S.queues.resize(n_media);
    cudaGetDevice(&S.device);
    {
        cudaError_t e = cudaStreamCreateWithFlags(&S.free_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            set_error(std::string("msp_server_create: stream: ") + cudaGetErrorString(e));
            return MSP_ERR_CUDA;
        }
    }
    for (int w = 0; w < n_workers; ++w) {
        auto* W = new Worker();
        cudaError_t e = cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete W;
            msp_server_destroy(h);
            set_error(std::string("msp_server_create: stream: ") + cudaGetErrorString(e));
            return MSP_ERR_CUDA;
        }
        S.workers.push_back(W);
    }
    for (Worker* W : S.workers) W->th = std::thread(worker_loop, &S, W);
    *out = h;
    return MSP_OK;
}

extern "C" msp_status msp_server_submit(msp_server h, int medium, const double* phi_host, uint64_t* req_id) {
    clear_error();
    MSP_CHECK_ARG(h && phi_host && req_id, "msp_server_submit: NULL argument");
    Server& S = h->S;
    MSP_CHECK_ARG(medium >= 0 && medium < (int)S.media.size(), "msp_server_submit: medium index out of range");
    if (S.request_bytes(medium) > S.budget) {
        set_error("msp_server_submit: one request of this medium needs more device memory than the budget");
        return MSP_ERR_OOM;
    }
    Request r;
    r.medium = medium;
    r.phi.assign(phi_host, phi_host + 4 * (size_t)S.media[medium]->N);
    r.t_submit = now_ms();
    std::lock_guard<std::mutex> lk(S.mu);
    const uint64_t id = S.next_id++;
    S.reqs.emplace(id, std::move(r));
    S.queues[medium].push_back(id);
    S.st.submitted += 1;
    *req_id = id;
    S.cv.notify_all();
    return MSP_OK;
}

extern "C" msp_status msp_server_poll(msp_server h, uint64_t req_id, int* done, double* latency_ms) {
    clear_error();
    MSP_CHECK_ARG(h && done, "msp_server_poll: NULL argument");
    Server& S = h->S;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(req_id);
    MSP_CHECK_ARG(it != S.reqs.end(), "msp_server_poll: unknown or released request");
    const Request& r = it->second;
    *done = r.state == 2 ? 1 : (r.state == -1 ? -1 : 0);
    if (latency_ms) *latency_ms = (r.state == 2 || r.state == -1) ? r.t_done - r.t_submit : -1.0;
    if (r.state == -1) {
        set_error("msp_server_poll: the request's batch failed");
        return r.status;
    }
    return MSP_OK;
}

extern "C" msp_status msp_server_fetch(msp_server h, uint64_t req_id, double* u_host) {
    clear_error();
    MSP_CHECK_ARG(h && u_host, "msp_server_fetch: NULL argument");
    Server& S = h->S;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.reqs.find(req_id);
    MSP_CHECK_ARG(it != S.reqs.end(), "msp_server_fetch: unknown or released request");
    MSP_CHECK_ARG(it->second.state == 2, "msp_server_fetch: the request is not done");
    const long long nn = (long long)(S.media[it->second.medium]->N + 1) * (S.media[it->second.medium]->N + 1);
    MSP_CUDA(cudaMemcpy(u_host, it->second.u, sizeof(double) * nn, cudaMemcpyDeviceToHost));
    release_locked(S, it);
    return MSP_OK;
}

extern "C" msp_status msp_server_release(msp_server h, uint64_t req_id) {
    clear_error();
    MSP_CHECK_ARG(h, "msp_server_release: NULL server");
    Server& S = h->S;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(req_id);
    MSP_CHECK_ARG(it != S.reqs.end(), "msp_server_release: unknown or released request");
    MSP_CHECK_ARG(it->second.state == 2 || it->second.state == -1, "msp_server_release: the request is not finished");
    release_locked(S, it);
    return MSP_OK;
}

extern "C" msp_status msp_server_step(msp_server h, void* stream, int* n_done) {
    clear_error();
    MSP_CHECK_ARG(h, "msp_server_step: NULL server");
    Server& S = h->S;
    MSP_CHECK_ARG(S.workers.empty(), "msp_server_step: the server runs worker threads");
    int medium = -1, engine = MSP_SERVE_MAP, it_max = 0;
    double it_tol = 0.0;
    std::vector<uint64_t> ids;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        admit(S, medium, ids);
        engine = S.engine;
        it_tol = S.it_tol;
        it_max = S.it_max_iter;
    }
    if (n_done) *n_done = 0;
    if (ids.empty()) return MSP_OK;
    msp_status st = run_batch(S, S.manual, (cudaStream_t)stream, medium, ids, engine, it_tol, it_max);
    if (st == MSP_OK && n_done) *n_done = (int)ids.size();
    return st;
}

extern "C" msp_status msp_server_set_engine(msp_server h, int engine, double tol, int max_iter) {
    clear_error();
    MSP_CHECK_ARG(h, "msp_server_set_engine: NULL server");
    MSP_CHECK_ARG(engine == MSP_SERVE_MAP || engine == MSP_SERVE_ITERATIVE_FP64, "msp_server_set_engine: unknown engine");
    Server& S = h->S;
    if (engine == MSP_SERVE_MAP) {
        for (Basis* b : S.media)
            MSP_CHECK_ARG(b->map_built, "msp_server_set_engine: the map engine needs msp_basis_build_map on every medium");
    } else {
        MSP_CHECK_ARG(tol > 0 && tol < 1 && max_iter >= 1, "msp_server_set_engine: tol in (0, 1), max_iter >= 1");
    }
    std::lock_guard<std::mutex> lk(S.mu);
    S.engine = engine;
    if (engine == MSP_SERVE_ITERATIVE_FP64) {
        S.it_tol = tol;
        S.it_max_iter = max_iter;
    }
    return MSP_OK;
}

extern "C" msp_status msp_server_get_stats(msp_server h, msp_server_stats* out) {
    clear_error();
    MSP_CHECK_ARG(h && out, "msp_server_get_stats: NULL argument");
    Server& S = h->S;
    std::lock_guard<std::mutex> lk(S.mu);
    *out = S.st;
    int queued = 0, in_flight = 0, held = 0;
    for (auto& kv : S.reqs) {
        if (kv.second.state == 0) ++queued;
        else if (kv.second.state == 1) ++in_flight;
        else ++held;
    }
    out->queued = queued;
    out->in_flight = in_flight;
    out->held = held;
    out->mem_in_use = S.mem_in_use;
    out->mem_peak = S.mem_peak;
    return MSP_OK;
}

extern "C" void msp_server_destroy(msp_server h) {
    if (!h) return;
    Server& S = h->S;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
    }
    S.cv.notify_all();
    for (Worker* W : S.workers) {
        if (W->th.joinable()) W->th.join();
    }
    for (auto& kv : S.reqs) {
        Request& r = kv.second;
        if (r.mem && --r.mem->refs == 0) {
            cudaFreeAsync(r.mem->u, S.free_stream);
            delete r.mem;
        }
        r.mem = nullptr;
    }
    for (Worker* W : S.workers) {
        free_worker(*W);
        delete W;
    }
    free_worker(S.manual);
    if (S.free_stream) {
        cudaStreamSynchronize(S.free_stream);
        cudaStreamDestroy(S.free_stream);
    }
    delete h;
}
