// C ABI of include/jk.h: argument checks, error reporting and the request
// server.  No exception crosses the boundary.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>

#include "plan.h"

namespace jk {
const char *last_error_str();
int finish_plan_device(Plan *P);
}  // namespace jk

struct jk_plan {
    jk::Plan *p;
    cudaEvent_t done;  // completion of the latest build on this plan (serialises builds across streams)
};

using jk::fail;

extern "C" {

const char *jk_status_string(int s)
{
    switch (s) {
    case JK_OK: return "ok";
    case JK_ERR_INVALID: return "invalid argument";
    case JK_ERR_UNSUPPORTED: return "unsupported (angular momentum above d)";
    case JK_ERR_OOM: return "out of memory or over budget";
    case JK_ERR_CUDA: return "CUDA or cuBLAS failure";
    case JK_ERR_TIMEOUT: return "timed out";
    case JK_ERR_DEVICE_CHECK: return "device-side bounds check tripped";
    case JK_ERR_BUSY: return "busy or shutting down";
    case JK_ERR_NOT_FOUND: return "unknown ticket";
    default: return "unknown status";
    }
}

const char *jk_last_error(void) { return jk::last_error_str(); }

int jk_plan_create(const jk_cell *cell, const jk_shell *shells, int nshell, double omega, const jk_cutoffs *cut,
                   jk_precision precision, int device, jk_plan **out)
{
    try {
        if (!out) return fail(JK_ERR_INVALID, "out is NULL");
        *out = nullptr;
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(JK_ERR_CUDA, "no CUDA device");
        if (device < 0 || device >= ndev) return fail(JK_ERR_INVALID, "device index out of range");
        jk::Plan *P = nullptr;
        int rc = jk::build_plan(cell, shells, nshell, omega, cut, precision, device, &P);
        if (rc) return rc;
        rc = jk::finish_plan_device(P);
        if (rc) {
            jk::destroy_plan(P);
            return rc;
        }
        jk_plan *h = new jk_plan{P, nullptr};
        if (cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess) {
            jk::destroy_plan(P);
            delete h;
            return fail(JK_ERR_CUDA, "cudaEventCreate failed");
        }
        cudaEventRecord(h->done, 0);
        *out = h;
        return JK_OK;
    } catch (const std::bad_alloc &) {
        return fail(JK_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(JK_ERR_INVALID, "unexpected host exception");
    }
}

int jk_pair_counts(const jk_cell *cell, const jk_shell *shells, int nshell, double omega, const jk_cutoffs *cut,
                   long long counts[5])
{
    if (!counts) return fail(JK_ERR_INVALID, "counts is NULL");
    try {
        jk::Plan *P = nullptr;
        int rc = jk::build_plan(cell, shells, nshell, omega, cut, JK_FP64, 0, &P);
        if (rc) return rc;
        counts[0] = P->n_ord_shell_pairs;
        counts[1] = P->n_ord_prim_pairs;
        counts[2] = P->n_ord_local_pairs;
        counts[3] = (long long)P->spi.size();
        counts[4] = (long long)(P->gvec.size() / 4);
        delete P;  // host part only: nothing was allocated on a device
        return JK_OK;
    } catch (const std::bad_alloc &) {
        return fail(JK_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(JK_ERR_INVALID, "unexpected host exception");
    }
}

int jk_plan_nbf(const jk_plan *plan) { return plan ? plan->p->nbf : -1; }

int jk_plan_info(const jk_plan *plan, jk_plan_stats *o)
{
    if (!plan || !o) return fail(JK_ERR_INVALID, "NULL argument");
    const jk::Plan *P = plan->p;
    *o = jk_plan_stats{};
    o->nbf = P->nbf;
    o->nshell = P->nshell;
    o->n_classes = 0;
    for (auto &c : P->classes) o->n_classes += c.b1 > c.b0;
    o->n_g = (int)(P->gvec.size() / 4);
    o->n_shell_pairs = P->n_shell_pairs;
    o->n_pair_images = (long long)P->spi.size();
    o->n_prim_pair_images = (long long)P->ppi.size();
    o->n_quartets = P->n_quartets;
    o->n_quartets_schwarz = P->n_quartets_schwarz;
    o->n_quartets_fp64 = P->n_quartets_fp64;
    o->n_r1_candidates = (long long)(P->r1.size() / 4);
    o->omega = P->omega;
    o->g_max = P->g_max;
    o->r1_max = P->r1_max;
    o->volume = P->volume;
    o->device_bytes = P->device_bytes + P->cache.bytes;
    o->workspace_bytes = P->ws.bytes;
    return JK_OK;
}

void jk_plan_destroy(jk_plan *plan)
{
    if (!plan) return;
    cudaSetDevice(plan->p->device);
    if (plan->done) {
        cudaEventSynchronize(plan->done);
        cudaEventDestroy(plan->done);
    }
    jk::destroy_plan(plan->p);
    delete plan;
}

int jk_build(jk_plan *plan, const double *D, double *J, double *K, void *cuda_stream)
{
    if (!plan || !D) return fail(JK_ERR_INVALID, "plan or D is NULL");
    if (!J && !K) return JK_OK;
    try {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        if (cudaSetDevice(plan->p->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
        // one critical section: order after the previous build on this plan,
        // enqueue, and publish this build's completion event, so builds from
        // several host threads on several streams run one after another on
        // the plan's single workspace
        std::lock_guard<std::mutex> g(plan->p->build_mu);
        cudaStreamWaitEvent(st, plan->done, 0);
        int rc = jk::run_build(plan->p, D, J, K, st);
        cudaEventRecord(plan->done, st);
        return rc;
    } catch (...) {
        return fail(JK_ERR_INVALID, "unexpected host exception");
    }
}

int jk_plan_cache(jk_plan *plan, size_t max_bytes, size_t *bytes)
{
    if (!plan) return fail(JK_ERR_INVALID, "plan is NULL");
    try {
        if (cudaSetDevice(plan->p->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
        std::lock_guard<std::mutex> g(plan->p->build_mu);
        // the cache may be in use by the plan's last build
        if (cudaEventSynchronize(plan->done) != cudaSuccess) return fail(JK_ERR_CUDA, "previous build failed");
        int rc = jk::cache_reciprocal(plan->p, max_bytes);
        if (bytes) *bytes = plan->p->cache.bytes;
        return rc;
    } catch (...) {
        return fail(JK_ERR_INVALID, "unexpected host exception");
    }
}

int jk_build_times(jk_plan *plan, double *ms, int *launches, int n)
{
    if (!plan || n < 0) return fail(JK_ERR_INVALID, "bad arguments");
    std::lock_guard<std::mutex> g(plan->p->build_mu);
    return jk::build_times(plan->p, ms, launches, n);
}

int jk_autotune(jk_plan *plan, const double *D, void *cuda_stream, const char *cache_path, int *chosen)
{
    if (!plan || !D) return fail(JK_ERR_INVALID, "plan or D is NULL");
    try {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        if (cudaSetDevice(plan->p->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
        std::lock_guard<std::mutex> g(plan->p->build_mu);
        cudaStreamWaitEvent(st, plan->done, 0);
        int rc = jk::autotune(plan->p, D, st, cache_path, chosen);
        cudaEventRecord(plan->done, st);
        return rc;
    } catch (...) {
        return fail(JK_ERR_INVALID, "unexpected host exception");
    }
}

int jk_plan_set_schedule(jk_plan *plan, const int *sched, int n)
{
    if (!plan || !sched || n < 0 || n > 21) return fail(JK_ERR_INVALID, "bad schedule arguments");
    std::lock_guard<std::mutex> g(plan->p->build_mu);
    return jk::set_schedule(plan->p, sched, n);
}

int jk_build_counts(jk_plan *plan, long long *counts, int n)
{
    if (!plan || !counts || n < 0) return fail(JK_ERR_INVALID, "bad arguments");
    std::lock_guard<std::mutex> g(plan->p->build_mu);
    return jk::build_counts(plan->p, counts, n);
}

int jk_build_host(jk_plan *plan, const double *Dh, double *Jh, double *Kh, void *cuda_stream)
{
    if (!plan || !Dh) return fail(JK_ERR_INVALID, "plan or D is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t bytes = sizeof(double) * plan->p->nbf * plan->p->nbf;
    if (cudaSetDevice(plan->p->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
    double *d = nullptr, *j = nullptr, *k = nullptr;
    if (cudaMallocAsync((void **)&d, bytes, st) != cudaSuccess || (Jh && cudaMallocAsync((void **)&j, bytes, st) != cudaSuccess) ||
        (Kh && cudaMallocAsync((void **)&k, bytes, st) != cudaSuccess)) {
        if (d) cudaFreeAsync(d, st);
        if (j) cudaFreeAsync(j, st);
        return fail(JK_ERR_OOM, "device buffers for host build");
    }
    int rc = JK_OK;
    if (cudaMemcpyAsync(d, Dh, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = fail(JK_ERR_CUDA, "copy of D failed");
    if (!rc) rc = jk_build(plan, d, j, k, cuda_stream);
    if (!rc && Jh && cudaMemcpyAsync(Jh, j, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = fail(JK_ERR_CUDA, "copy of J failed");
    if (!rc && Kh && cudaMemcpyAsync(Kh, k, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = fail(JK_ERR_CUDA, "copy of K failed");
    cudaFreeAsync(d, st);
    if (j) cudaFreeAsync(j, st);
    if (k) cudaFreeAsync(k, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = fail(JK_ERR_CUDA, "host build failed");
    return rc;
}

__global__ void jk_energy_kernel(size_t n2, const double *D, const double *J, const double *K, double *out);

int jk_energy(const jk_plan *plan, const double *D, const double *J, const double *K, double *e_coul, double *e_exch, void *cuda_stream)
{
    if (!plan || !D || !e_coul || !e_exch) return fail(JK_ERR_INVALID, "NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(plan->p->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
    const size_t n2 = (size_t)plan->p->nbf * plan->p->nbf;
    double *dev = nullptr;
    if (cudaMallocAsync((void **)&dev, 2 * sizeof(double), st) != cudaSuccess) return fail(JK_ERR_OOM, "energy scratch");
    cudaMemsetAsync(dev, 0, 2 * sizeof(double), st);
    jk_energy_kernel<<<(unsigned)std::min<size_t>((n2 + 255) / 256, 2432), 256, 0, st>>>(n2, D, J, K, dev);
    double h[2] = {0, 0};
    cudaMemcpyAsync(h, dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dev, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(JK_ERR_CUDA, "energy reduction failed");
    *e_coul = 0.5 * h[0];
    *e_exch = -0.25 * h[1];
    return JK_OK;
}

int jk_energy_noalloc(const jk_plan *plan, const double *D, const double *J, const double *K, double *e_coul, double *e_exch,
                      void *cuda_stream)
{
    if (!plan || !D || !e_coul || !e_exch) return fail(JK_ERR_INVALID, "NULL argument");
    return jk::energy_noalloc(plan->p, D, J, K, e_coul, e_exch, (cudaStream_t)cuda_stream);
}

__global__ void jk_scale_kernel(int n, const double *f, const double *A, double *B);

int jk_overlap(const jk_plan *plan, double *S, void *cuda_stream)
{
    if (!plan || !S) return fail(JK_ERR_INVALID, "NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(plan->p->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
    const size_t n2 = (size_t)plan->p->nbf * plan->p->nbf;
    jk_scale_kernel<<<(unsigned)std::min<size_t>((n2 + 255) / 256, 2432), 256, 0, st>>>(plan->p->nbf, plan->p->d_compf, plan->p->d_S, S);
    if (cudaGetLastError() != cudaSuccess) return fail(JK_ERR_CUDA, "overlap kernel failed");
    return JK_OK;
}

int jk_one_electron(jk_plan *plan, int natom, const double *Z, const double *xyz, double *T, double *V, void *cuda_stream)
{
    if (!plan || natom < 0 || (V && natom > 0 && (!Z || !xyz))) return fail(JK_ERR_INVALID, "bad one-electron arguments");
    try {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        if (cudaSetDevice(plan->p->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
        std::lock_guard<std::mutex> g(plan->p->build_mu);
        cudaStreamWaitEvent(st, plan->done, 0);
        int rc = jk::one_electron(plan->p, natom, Z, xyz, T, V, st);
        cudaEventRecord(plan->done, st);
        return rc;
    } catch (...) {
        return fail(JK_ERR_INVALID, "unexpected host exception");
    }
}

int jk_ewald_point_charges(const jk_cell *cell, int n, const double *q, const double *xyz, double omega, double delta, double *energy)
{
    if (!cell || !q || !xyz || !energy || n <= 0 || !(omega > 0)) return fail(JK_ERR_INVALID, "bad point-charge arguments");
    *energy = jk::ewald_point_charges_host(cell->lattice, n, q, xyz, omega, delta > 0 ? delta : 1e-14);
    return JK_OK;
}

}  // extern "C"

__global__ void jk_energy_kernel(size_t n2, const double *D, const double *J, const double *K, double *out)
{
    double s0 = 0, s1 = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        if (J) s0 += D[i] * J[i];
        if (K) s1 += D[i] * K[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    __shared__ double sh[2][32];
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        atomicAdd(out, a);
        atomicAdd(out + 1, b);
    }
}

__global__ void jk_scale_kernel(int n, const double *f, const double *A, double *B)
{
    const size_t n2 = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x)
        B[i] = f[i / n] * f[i % n] * A[i];
}

// ---------------------------------------------------------------------------
// Request server: continuous batching of builds.  A scheduler thread admits
// queued requests in arrival order whenever a slot (stream) is free and the
// workspace of the plans in flight plus the candidate's stays within the HBM
// budget; completion is detected with events, so requests that arrive while
// others run are admitted as soon as room frees up and their kernels overlap
// on the device.
namespace {
struct Request {
    long long ticket;
    jk_plan *plan;
    const double *D;
    double *J, *K;
    std::chrono::steady_clock::time_point t_submit;
};
struct Done {
    int status;
    double latency;
};
struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    Request req{};
    int status = 0;
    size_t bytes = 0;
};
}  // namespace

struct jk_server {
    int device = 0;
    size_t budget = 0;
    std::vector<Slot> slots;
    std::deque<Request> pending;
    std::map<long long, Done> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stopping = false;
    long long next_ticket = 1;
    size_t in_flight_bytes = 0;
    std::atomic<int> in_flight{0};

    void loop()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            // retire finished slots
            for (auto &s : slots) {
                if (!s.busy) continue;
                if (cudaEventQuery(s.ev) == cudaSuccess) {
                    double lat = std::chrono::duration<double>(std::chrono::steady_clock::now() - s.req.t_submit).count();
                    done[s.req.ticket] = Done{s.status, lat};
                    s.busy = false;
                    in_flight_bytes -= s.bytes;
                    in_flight--;
                    cv_done.notify_all();
                }
            }
            // admit in arrival order
            while (!pending.empty()) {
                Slot *free_slot = nullptr;
                for (auto &s : slots)
                    if (!s.busy) {
                        free_slot = &s;
                        break;
                    }
                if (!free_slot) break;
                const Request &r = pending.front();
                size_t need = r.plan->p->ws.bytes;
                if (in_flight_bytes + need > budget && in_flight > 0) break;  // wait for memory to free up
                Request req = pending.front();
                pending.pop_front();
                free_slot->req = req;
                free_slot->bytes = need;
                free_slot->busy = true;
                in_flight_bytes += need;
                in_flight++;
                lk.unlock();
                int st = jk_build(req.plan, req.D, req.J, req.K, free_slot->st);
                cudaEventRecord(free_slot->ev, free_slot->st);
                lk.lock();
                free_slot->status = st;
            }
            if (stopping && pending.empty() && in_flight == 0) break;
            cv_work.wait_for(lk, std::chrono::microseconds(in_flight > 0 ? 50 : 2000));
        }
    }
};

extern "C" {

int jk_server_create(int device, size_t hbm_budget_bytes, int max_slots, jk_server **out)
{
    if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return fail(JK_ERR_INVALID, "bad server arguments");
    *out = nullptr;
    try {
        jk_server *s = new jk_server();
        s->device = device;
        s->budget = hbm_budget_bytes;
        if (cudaSetDevice(device) != cudaSuccess) {
            delete s;
            return fail(JK_ERR_CUDA, "cudaSetDevice failed");
        }
        s->slots.resize(max_slots);
        for (auto &sl : s->slots) {
            if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
                for (auto &x : s->slots) {
                    if (x.st) cudaStreamDestroy(x.st);
                    if (x.ev) cudaEventDestroy(x.ev);
                }
                delete s;
                return fail(JK_ERR_CUDA, "stream creation failed");
            }
        }
        s->worker = std::thread([s] { s->loop(); });
        *out = s;
        return JK_OK;
    } catch (...) {
        return fail(JK_ERR_OOM, "server allocation failed");
    }
}

int jk_submit(jk_server *srv, jk_plan *plan, const double *D, double *J, double *K, long long *ticket)
{
    if (!srv || !plan || !D || !ticket) return fail(JK_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return fail(JK_ERR_BUSY, "server is shutting down");
    if (plan->p->ws.bytes > srv->budget) return fail(JK_ERR_OOM, "plan workspace exceeds the server's HBM budget");
    Request r{srv->next_ticket++, plan, D, J, K, std::chrono::steady_clock::now()};
    srv->pending.push_back(r);
    *ticket = r.ticket;
    srv->cv_work.notify_one();
    return JK_OK;
}

int jk_wait(jk_server *srv, long long ticket, int timeout_ms, int *build_status, double *latency_s)
{
    if (!srv) return fail(JK_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] { return srv->done.count(ticket) > 0; };
    auto known = [&] {
        if (ready()) return true;
        for (auto &r : srv->pending)
            if (r.ticket == ticket) return true;
        for (auto &s : srv->slots)
            if (s.busy && s.req.ticket == ticket) return true;
        return false;
    };
    if (!known()) return fail(JK_ERR_NOT_FOUND, "unknown or already collected ticket");
    if (timeout_ms < 0)
        srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(JK_ERR_TIMEOUT, "ticket not finished");
    Done d = srv->done[ticket];
    srv->done.erase(ticket);
    if (build_status) *build_status = d.status;
    if (latency_s) *latency_s = d.latency;
    return JK_OK;
}

void jk_server_destroy(jk_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->device);
    for (auto &s : srv->slots) {
        if (s.st) {
            cudaStreamSynchronize(s.st);
            cudaStreamDestroy(s.st);
        }
        if (s.ev) cudaEventDestroy(s.ev);
    }
    delete srv;
}

}  // extern "C"
