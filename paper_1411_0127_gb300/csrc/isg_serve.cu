// isg_serve.cu -- request server: quench jobs of mixed L, sweep count, T and
// generator, served by continuous batching on one GPU.
//
// A job is one lattice (isg_create arguments) and a number of sweeps.  Jobs are
// submitted with an arrival time (seconds after the start of isg_server_run);
// the run loop is:
//   1. admit, in arrival order, the jobs that have arrived while the device
//      memory they need fits the budget and a slot is free (a job that does not
//      fit blocks the ones behind it: first come, first served);
//   2. run one quantum: every active lattice's streams become items of the
//      pass engine (one launch per colour pass and generator kind, 4-warp CTAs
//      taking (lattice, stream) items by ticket, longest first), each lattice
//      running min(quantum, sweeps left) sweeps; the three kinds' launches run
//      on streams of their own;
//   3. retire the jobs that are done: energy from scratch and Zobrist hash,
//      completion time, memory returned to the budget.
// The lattices, couplings and generator states stay on the device between
// quanta.  A lattice's trajectory depends only on its own seeds and on how many
// sweeps it has had, never on which jobs shared a launch with it, so a job's
// result is the same alone and in any mix (checked by the tests).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "isg_bundles.cuh"

namespace isg {

constexpr int kKinds = 3;   // generator kinds: one bundle plan and stream each

struct ServeJob {
    int L = 0, kind = 0;
    uint64_t seed_J = 0, seed_spin = 0;
    double beta = 0.0, arrival = 0.0;
    int64_t sweeps = 0, done = 0;
    isg_sim* h = nullptr;
    size_t bytes = 0;
    int status = 0;  // 0 waiting, 1 active, 2 finished, < 0 failed (ISG_ERR_*)
    double t_admit = -1.0, t_done = -1.0;
    int64_t E = 0;
    uint64_t H = 0;
};

struct PlanBuf {
    FlipArgs* reps = nullptr;
    int2* items = nullptr;
    int* limit = nullptr;
    unsigned* ctr = nullptr;
    size_t cap_reps = 0, cap_items = 0, cap_limit = 0;
    // host copies of the current plan (alive until the quantum has finished)
    std::vector<FlipArgs> desc;
    std::vector<int2> h_items;
    std::vector<int> h_limit, idx;
    std::vector<int64_t> give;
};

}  // namespace isg

struct isg_server {
    size_t budget = 0;
    int quantum = 64;
    int max_active = 4096;
    std::mutex mu;
    std::vector<isg::ServeJob> jobs;
    isg::PlanBuf plan[isg::kKinds];
    cudaStream_t batch_stream[isg::kKinds] = {nullptr, nullptr, nullptr};
    // statistics of the last run
    int64_t iterations = 0, attempts = 0;
    double wall = 0.0, busy = 0.0;
    int peak_active = 0;
    size_t peak_bytes = 0;
};

namespace isg {

static double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

static void* g_dev_alloc(size_t n) {
    void* p = nullptr;
    return cudaMalloc(&p, n) == cudaSuccess ? p : nullptr;
}

// Grow a device buffer to hold `need` elements of size `elem`.
template <typename T>
static bool ensure(T*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return true;
    size_t c = std::max<size_t>(need, 2 * cap + 64);
    if (p) cudaFree(p);
    p = (T*)g_dev_alloc(c * sizeof(T));
    cap = p ? c : 0;
    return p != nullptr;
}

// Enqueue one quantum of the batched jobs of one generator kind: every stream
// of every such job is an item of the pass engine, longest streams first; job j
// runs give_j = min(quantum, sweeps left) sweeps, so its items take part in the
// first 2 give_j of the 2 max(give) pass launches.  The plan's host copies stay
// in s->plan[kind] until finish_batched has run.
static int launch_batched(isg_server* s, int kind, const std::vector<int>& active) {
    PlanBuf& P = s->plan[kind];
    P.idx.clear();
    P.desc.clear();
    P.h_limit.clear();
    P.h_items.clear();
    P.give.clear();
    int64_t qmax = 0;
    for (int j : active) {
        const ServeJob& J = s->jobs[j];
        if (J.kind != kind) continue;
        const int64_t q = std::min<int64_t>(s->quantum, J.sweeps - J.done);
        const int r = (int)P.idx.size();
        P.idx.push_back(j);
        P.give.push_back(q);
        P.desc.push_back(make_flip_args(J.h, 0));
        P.h_limit.push_back((int)(2 * q));
        for (int64_t t = 0; t < J.h->S; ++t) P.h_items.push_back(make_int2(r, (int)t));
        qmax = std::max(qmax, q);
    }
    if (P.idx.empty() || qmax == 0) return ISG_OK;
    auto draws = [&](const int2& it) {
        const isg_sim* h = s->jobs[P.idx[it.x]].h;
        const int64_t r0 = (int64_t)it.y * h->R, r1 = std::min(r0 + h->R, h->rows);
        return (r1 - r0) * h->half;
    };
    std::stable_sort(P.h_items.begin(), P.h_items.end(),
                     [&](const int2& x, const int2& y) { return draws(x) > draws(y); });
    if (!ensure(P.reps, P.cap_reps, P.desc.size()) || !ensure(P.items, P.cap_items, P.h_items.size()) ||
        !ensure(P.limit, P.cap_limit, P.h_limit.size())) {
        set_error("isg_server_run: device allocation for the quantum plan failed");
        return ISG_ERR_NOMEM;
    }
    cudaStream_t st = s->batch_stream[kind];
    cudaError_t e =
        cudaMemcpyAsync(P.reps, P.desc.data(), P.desc.size() * sizeof(FlipArgs), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.items, P.h_items.data(), P.h_items.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.limit, P.h_limit.data(), P.h_limit.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_pass_items(kind, P.reps, P.items, (int)P.h_items.size(), P.limit, (int)qmax, P.ctr, st);
    if (e != cudaSuccess) return cuda_fail(e, "isg_server_run: batched quantum");
    return ISG_OK;
}

// After the quantum's streams have finished: credit the sweeps to the jobs.
static int finish_batched(isg_server* s, int kind) {
    PlanBuf& P = s->plan[kind];
    const cudaError_t e = cudaStreamSynchronize(s->batch_stream[kind]);
    if (e != cudaSuccess) return cuda_fail(e, "isg_server_run: batched quantum");
    for (size_t r = 0; r < P.idx.size(); ++r) {
        ServeJob& J = s->jobs[P.idx[r]];
        J.done += P.give[r];
        J.h->sweeps += P.give[r];
        J.h->last_stream = s->batch_stream[kind];
        s->attempts += P.give[r] * (int64_t)J.L * J.L * J.L;
    }
    P.idx.clear();
    P.give.clear();
    return ISG_OK;
}

}  // namespace isg

using namespace isg;

extern "C" {

int isg_server_create(size_t hbm_budget_bytes, int quantum_sweeps, int max_active, isg_server** out) {
    if (!out || hbm_budget_bytes == 0) { set_error("isg_server_create: bad argument"); return ISG_ERR_ARG; }
    *out = nullptr;
    isg_server* s = new (std::nothrow) isg_server();
    if (!s) { set_error("isg_server_create: out of host memory"); return ISG_ERR_NOMEM; }
    s->budget = hbm_budget_bytes;
    s->quantum = quantum_sweeps > 0 ? quantum_sweeps : 64;
    s->max_active = max_active > 0 ? max_active : 4096;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kKinds && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->batch_stream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            s->plan[k].ctr = (unsigned*)g_dev_alloc(3 * sizeof(unsigned));
            if (!s->plan[k].ctr) e = cudaErrorMemoryAllocation;
        }
        if (e == cudaSuccess) e = cudaMemset(s->plan[k].ctr, 0, 3 * sizeof(unsigned));
    }
    if (e != cudaSuccess) {
        isg_server_destroy(s);
        return cuda_fail(e, "isg_server_create");
    }
    *out = s;
    return ISG_OK;
}

void isg_server_destroy(isg_server* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    for (ServeJob& J : s->jobs)
        if (J.h) destroy_sim(J.h);
    for (PlanBuf& P : s->plan) {
        cudaFree(P.reps);
        cudaFree(P.items);
        cudaFree(P.limit);
        cudaFree(P.ctr);
    }
    for (cudaStream_t st : s->batch_stream)
        if (st) cudaStreamDestroy(st);
    delete s;
}

int isg_server_submit(isg_server* s, int L, uint64_t seed_J, uint64_t seed_spin, double beta, int rng_kind,
                      int64_t sweeps, double arrival_s, int64_t* job_id) {
    if (!s || !job_id || sweeps < 0 || L < 4 || L > 2048 || (L & 1) || !(beta > 0.0) ||
        !rng_kind_valid(rng_kind) || !(arrival_s >= 0.0)) {
        set_error("isg_server_submit: bad argument (L=%d beta=%g kind=%d sweeps=%lld)", L, beta, rng_kind,
                  (long long)sweeps);
        return ISG_ERR_ARG;
    }
    ServeJob J;
    J.L = L;
    J.kind = rng_kind;
    J.seed_J = seed_J;
    J.seed_spin = seed_spin;
    J.beta = beta;
    J.sweeps = sweeps;
    J.arrival = arrival_s;
    J.bytes = sim_device_bytes(L, rng_kind, true);
    if (J.bytes > s->budget) {
        set_error("isg_server_submit: job needs %zu bytes, the budget is %zu", J.bytes, s->budget);
        return ISG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *job_id = (int64_t)s->jobs.size();
    s->jobs.push_back(J);
    return ISG_OK;
}

int isg_server_run(isg_server* s, double time_limit_s) {
    if (!s) { set_error("isg_server_run: NULL server"); return ISG_ERR_ARG; }
    std::vector<int> order;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int j = 0; j < (int)s->jobs.size(); ++j)
            if (s->jobs[j].status == 0) order.push_back(j);
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return s->jobs[a].arrival < s->jobs[b].arrival; });
    const auto t0 = std::chrono::steady_clock::now();
    s->iterations = 0;
    s->attempts = 0;
    s->busy = 0.0;
    s->peak_active = 0;
    s->peak_bytes = 0;
    size_t next = 0, used = 0;
    int64_t remaining = (int64_t)order.size();
    std::vector<int> active;
    while (remaining > 0) {
        double now = now_s(t0);
        if (time_limit_s > 0.0 && now > time_limit_s) {
            set_error("isg_server_run: time limit of %g s reached with %lld jobs unfinished", time_limit_s,
                      (long long)remaining);
            return ISG_ERR_TIMEOUT;
        }
        // 1. admission, first come first served
        while (next < order.size()) {
            ServeJob& J = s->jobs[order[next]];
            if (J.arrival > now || used + J.bytes > s->budget || (int)active.size() >= s->max_active) break;
            const int rc = create_sim(J.L, J.seed_J, J.seed_spin, J.seed_spin, J.beta, J.kind, true, &J.h);
            ++next;
            if (rc) {
                J.status = rc;
                J.t_done = now_s(t0);
                --remaining;
                continue;
            }
            J.status = 1;
            J.t_admit = now_s(t0);
            used += J.bytes;
            active.push_back(order[next - 1]);
        }
        s->peak_active = std::max(s->peak_active, (int)active.size());
        s->peak_bytes = std::max(s->peak_bytes, used);
        if (active.empty()) {
            if (next < order.size()) {
                const double wait = s->jobs[order[next]].arrival - now_s(t0);
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
            }
            continue;
        }
        // 2. one quantum: per generator kind, pass launches over all its jobs' streams
        const double tq = now_s(t0);
        for (int k = 0; k < kKinds; ++k) {
            const int rc = launch_batched(s, k, active);
            if (rc) return rc;
        }
        for (int k = 0; k < kKinds; ++k) {
            const int rc = finish_batched(s, k);
            if (rc) return rc;
        }
        s->busy += now_s(t0) - tq;
        ++s->iterations;
        // 3. retire finished jobs
        std::vector<int> still;
        for (int j : active) {
            ServeJob& J = s->jobs[j];
            if (J.done < J.sweeps) {
                still.push_back(j);
                continue;
            }
            int rc = isg_energy(J.h, &J.E, s->batch_stream[0]);
            if (!rc) rc = isg_hash(J.h, &J.H, s->batch_stream[0]);
            J.t_done = now_s(t0);
            J.status = rc ? rc : 2;
            destroy_sim(J.h);
            J.h = nullptr;
            used -= J.bytes;
            --remaining;
        }
        active.swap(still);
    }
    s->wall = now_s(t0);
    return ISG_OK;
}

int isg_server_job(const isg_server* s, int64_t id, int* status, int64_t* E, uint64_t* H, double* arrival_s,
                   double* admit_s, double* done_s) {
    if (!s || id < 0 || id >= (int64_t)s->jobs.size()) { set_error("isg_server_job: bad job id"); return ISG_ERR_ARG; }
    const ServeJob& J = s->jobs[id];
    if (status) *status = J.status;
    if (E) *E = J.E;
    if (H) *H = J.H;
    if (arrival_s) *arrival_s = J.arrival;
    if (admit_s) *admit_s = J.t_admit;
    if (done_s) *done_s = J.t_done;
    return ISG_OK;
}

int isg_server_stats(const isg_server* s, int64_t* iterations, int64_t* attempts, double* wall_s, double* busy_s,
                     int* peak_active, size_t* peak_bytes) {
    if (!s) { set_error("isg_server_stats: NULL server"); return ISG_ERR_ARG; }
    if (iterations) *iterations = s->iterations;
    if (attempts) *attempts = s->attempts;
    if (wall_s) *wall_s = s->wall;
    if (busy_s) *busy_s = s->busy;
    if (peak_active) *peak_active = s->peak_active;
    if (peak_bytes) *peak_bytes = s->peak_bytes;
    return ISG_OK;
}

}  // extern "C"
