// isg_api.cu -- the extern "C" boundary (include/isg.h): argument checks,
// allocation through the installed allocator, kernel launches, status codes.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "isg_common.cuh"

namespace isg {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return ISG_ERR_CUDA;
}

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    return dev < 0 ? 0 : dev;
}

int sm_count() {
    static std::atomic<int> cache[kDeviceSlots];
    const int dev = current_device();
    if (dev < kDeviceSlots) {
        const int v = cache[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    if (dev < kDeviceSlots) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

static void* default_alloc(size_t n, void*) {
    void* p = nullptr;
    return cudaMalloc(&p, n) == cudaSuccess ? p : nullptr;
}
static void default_free(void* p, void*) { cudaFree(p); }

static std::mutex g_alloc_mu;
static void* (*g_alloc)(size_t, void*) = default_alloc;
static void (*g_free)(void*, void*) = default_free;
static void* g_alloc_ctx = nullptr;

void* dev_alloc(isg_sim* h, size_t n) { return h->alloc(n ? n : 1, h->alloc_ctx); }
void dev_free(isg_sim* h, void* p) {
    if (p) h->free_fn(p, h->alloc_ctx);
}

// floor(2^32 exp(-4 k beta)), k = 1..3 (Sec. 4, Rmax exp(-beta dE)).
void thresholds(double beta, uint32_t thr[4]) {
    thr[0] = 0;
    for (int k = 1; k <= 3; ++k) {
        const double v = std::floor(4294967296.0 * std::exp(-4.0 * k * beta));
        thr[k] = v <= 0.0 ? 0u : (v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v);
    }
}

// Stream partition: S0 = clamp(L^3 / 32768, 1, 8192); R = ceil(L^2 / S0).
static void partition(int L, int64_t* R, int64_t* S) {
    const int64_t rows = (int64_t)L * L;
    int64_t s0 = (int64_t)L * L * L / 32768;
    s0 = s0 < 1 ? 1 : (s0 > 8192 ? 8192 : s0);
    *R = (rows + s0 - 1) / s0;
    *S = (rows + *R - 1) / *R;
}

static bool beta_ok(double beta) { return beta > 0.0; }  // false for 0, negatives, NaN

// Fill the geometry fields and allocate every device buffer (zeroed).
static int alloc_sim(isg_sim* h) {
    h->half = h->L / 2;
    const int w64 = (h->half + 63) / 64, w32 = (h->half + 31) / 32;
    // 64-bit words where they waste no more bits than 32-bit ones; batch members
    // always use them (one kernel instantiation serves every size of a batch)
    h->wbits = (h->member || 2 * w64 == w32) ? 64 : 32;
    h->W = (h->half + h->wbits - 1) / h->wbits;
    h->nt = h->half - (h->W - 1) * h->wbits;
    h->rows = (int64_t)h->L * h->L;
    partition(h->L, &h->R, &h->S);
    const int64_t raw = h->rows * h->W * (h->wbits / 8);
    h->plane_bytes = (raw + 255) / 256 * 256;
    const size_t pbytes = (size_t)h->plane_bytes * 8;
    h->planes = (unsigned char*)dev_alloc(h, pbytes);
    const size_t rng_words = (size_t)h->S * rng_state_words(h->kind);
    h->rng = (uint32_t*)dev_alloc(h, rng_words * 4);
    h->rng_pos = (uint32_t*)dev_alloc(h, (size_t)h->S * 4);
    if (h->kind == ISG_RNG_MINSTD) h->rng_alt = (uint32_t*)dev_alloc(h, rng_words * 4);
    h->scal = (long long*)dev_alloc(h, 8 * sizeof(long long));
    if (!h->member) h->done = (unsigned long long*)dev_alloc(h, (size_t)h->S * sizeof(unsigned long long));
    if (!h->planes || !h->rng || !h->rng_pos || !h->scal || (h->kind == ISG_RNG_MINSTD && !h->rng_alt) ||
        (!h->member && !h->done)) {
        set_error("isg: device allocation failed (%zu bytes of planes)", pbytes);
        return ISG_ERR_NOMEM;
    }
    cudaError_t e = cudaMemset(h->planes, 0, pbytes);
    if (e == cudaSuccess) e = cudaMemset(h->scal, 0, 8 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(h->rng_pos, 0, (size_t)h->S * 4);
    if (e == cudaSuccess && h->done) e = cudaMemset(h->done, 0, (size_t)h->S * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    return ISG_OK;
}

static void free_sim(isg_sim* h) {
    if (!h) return;
    dev_free(h, h->planes);
    dev_free(h, h->rng);
    dev_free(h, h->rng_pos);
    dev_free(h, h->rng_alt);
    dev_free(h, h->scal);
    dev_free(h, h->done);
    dev_free(h, h->stage);
    delete h;
}

static isg_sim* new_sim() {
    isg_sim* h = new (std::nothrow) isg_sim();
    if (!h) return nullptr;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h->alloc = g_alloc;
    h->free_fn = g_free;
    h->alloc_ctx = g_alloc_ctx;
    return h;
}

// Energy from scratch into *E, on stream s (sync).
// ISG_ERR_TIMEOUT (once: the word is cleared) if the handle's error word scal[5]
// is set: a bounded wait of a multi-pass sweep launch gave up, so passes were
// skipped and the configuration is no longer on its trajectory.
static int wait_error(const isg_sim* h, long long word, cudaStream_t s) {
    if (word == 0) return ISG_OK;
    const cudaError_t e = cudaMemsetAsync(h->scal + 5, 0, sizeof(long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the error word");
    set_error("a bounded wait of a multi-pass sweep launch gave up: passes were skipped");
    return ISG_ERR_TIMEOUT;
}

static int energy_sync(const isg_sim* h, int64_t* E, cudaStream_t s) {
    long long* acc = h->scal + 1;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = launch_energy(h, acc, s);
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel launch");
    long long w[5] = {0, 0, 0, 0, 0};  // scal[1..5]: U, ..., the error word
    e = cudaMemcpyAsync(w, acc, sizeof w, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "energy");
    if (const int rc = wait_error(h, w[4], s)) return rc;
    *E = 2 * (int64_t)w[0] - 3 * (int64_t)h->L * h->L * h->L;
    return ISG_OK;
}

// Tracking restart on the device (isg_exchange_async): dE := E(now) - E0, so
// that E0 + dE stays the tracked energy with the host's E0 untouched.
__global__ void restart_on_device_kernel(long long* scal, long long threeN, long long E0) {
    scal[0] = 2 * scal[1] - threeN - E0;
}

// The same restart folded into the first colour pass after new spins came in:
// that pass counted the configuration's unsatisfied bonds U into scal[1] before
// its flips and their dE into scal[0], so dE := dE + E(before the pass) - E0.
__global__ void restart_after_pass_kernel(long long* scal, long long threeN, long long E0) {
    scal[0] += 2 * scal[1] - threeN - E0;
}

// scal[4] = E0 + dE, the tracked energy, for an asynchronous read.
__global__ void tracked_word_kernel(long long* scal, long long E0) { scal[4] = E0 + scal[0]; }

// Restart the energy bookkeeping from the current configuration.
static int restart_tracking(isg_sim* h, cudaStream_t s) {
    int rc = energy_sync(h, &h->E0, s);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(h->scal, 0, sizeof(long long), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "reset tracked energy");
}

int create_sim(int L, uint64_t seed_J, uint64_t seed_spin, uint64_t seed_rng, double beta, int rng_kind, bool member,
               isg_sim** out) {
    if (!out) { set_error("isg_create: out is NULL"); return ISG_ERR_ARG; }
    *out = nullptr;
    if (L < 4 || L > 2048 || (L & 1)) { set_error("isg_create: L=%d must be even and in [4, 2048]", L); return ISG_ERR_ARG; }
    if (!beta_ok(beta)) { set_error("isg_create: beta must be > 0 (got %g)", beta); return ISG_ERR_ARG; }
    if (!rng_kind_valid(rng_kind)) {
        set_error("isg_create: unknown rng_kind %d", rng_kind);
        return ISG_ERR_ARG;
    }
    isg_sim* h = new_sim();
    if (!h) { set_error("isg_create: out of host memory"); return ISG_ERR_NOMEM; }
    h->L = L;
    h->kind = rng_kind;
    h->beta = beta;
    h->seed_J = seed_J;
    h->seed_spin = seed_spin;
    h->seed_rng = seed_rng;
    h->member = member;
    thresholds(beta, h->thr);
    int rc = alloc_sim(h);
    if (rc) { free_sim(h); return rc; }
    cudaError_t e = launch_init_planes(h, 0);
    if (e == cudaSuccess) e = launch_init_rng(h, 0);
    if (e != cudaSuccess) { free_sim(h); return cuda_fail(e, "init kernels"); }
    rc = restart_tracking(h, 0);
    if (rc) { free_sim(h); return rc; }
    *out = h;
    return ISG_OK;
}

void destroy_sim(isg_sim* h) { free_sim(h); }

// Device bytes a handle of this size and kind holds (planes, streams, words).
size_t sim_device_bytes(int L, int rng_kind, bool member) {
    const int half = L / 2;
    const int w64 = (half + 63) / 64, w32 = (half + 31) / 32;
    const int wbits = (member || 2 * w64 == w32) ? 64 : 32;
    const int W = (half + wbits - 1) / wbits;
    const int64_t rows = (int64_t)L * L;
    int64_t R = 0, S = 0;
    partition(L, &R, &S);
    const int64_t plane = (rows * W * (wbits / 8) + 255) / 256 * 256;
    const int64_t rng = S * rng_state_words(rng_kind) * 4 * (rng_kind == ISG_RNG_MINSTD ? 2 : 1);
    const int64_t done = member ? 0 : S * (int64_t)sizeof(unsigned long long);
    return (size_t)(8 * plane + rng + S * 4 + 8 * (int64_t)sizeof(long long) + done);
}

}  // namespace isg

using namespace isg;

extern "C" {

const char* isg_last_error(void) { return g_err; }

int isg_set_allocator(void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*), void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("isg_set_allocator: give both functions or neither");
        return ISG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc ? alloc : default_alloc;
    g_free = free_fn ? free_fn : default_free;
    g_alloc_ctx = alloc ? ctx : nullptr;
    return ISG_OK;
}

int isg_create(int L, uint64_t seed_J, uint64_t seed_spin, double beta, int rng_kind, isg_sim** out) {
    return create_sim(L, seed_J, seed_spin, seed_spin, beta, rng_kind, false, out);
}

int isg_create2(int L, uint64_t seed_J, uint64_t seed_spin, uint64_t seed_rng, double beta, int rng_kind,
                isg_sim** out) {
    return create_sim(L, seed_J, seed_spin, seed_rng, beta, rng_kind, false, out);
}

void isg_destroy(isg_sim* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_sim(h);
}

int isg_info(const isg_sim* h, int* L, int* word_bits, int* words_per_row, int64_t* streams,
             int64_t* rows_per_stream) {
    if (!h) { set_error("isg_info: NULL handle"); return ISG_ERR_ARG; }
    if (L) *L = h->L;
    if (word_bits) *word_bits = h->wbits;
    if (words_per_row) *words_per_row = h->W;
    if (streams) *streams = h->S;
    if (rows_per_stream) *rows_per_stream = h->R;
    return ISG_OK;
}

int isg_sweep_plain(isg_sim* h, int64_t n, void* stream) {
    if (!h || n < 0) { set_error("isg_sweep_plain: bad handle or n"); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = launch_flip_plain(h, 0, s);
        if (e == cudaSuccess) e = launch_flip_plain(h, 1, s);
        if (e != cudaSuccess) return cuda_fail(e, "flip kernel launch");
    }
    h->sweeps += n;
    h->last_stream = s;
    return ISG_OK;
}

int isg_sweep(isg_sim* h, int64_t n, void* stream) {
    if (!h || n < 0) { set_error("isg_sweep: bad handle or n"); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (sweeps_in_one_launch(h, n)) {
        // enough streams and sweeps: all passes in persistent launches of up to 64 sweeps
        const cudaError_t e = launch_sweeps(h, n, s);
        if (e != cudaSuccess) return cuda_fail(e, "sweep kernel launch");
    } else {
        for (int64_t k = 0; k < n; ++k) {
            cudaError_t e = launch_flip_fast(h, 0, s);
            if (e == cudaSuccess) e = launch_flip_fast(h, 1, s);
            if (e != cudaSuccess) return cuda_fail(e, "flip kernel launch");
        }
    }
    h->sweeps += n;
    h->last_stream = s;
    return ISG_OK;
}

int isg_sweep_info(const isg_sim* h, int* passes_per_launch) {
    if (!h || !passes_per_launch) { set_error("isg_sweep_info: NULL argument"); return ISG_ERR_ARG; }
    *passes_per_launch = sweeps_in_one_launch(h, 64) ? 128 : 1;
    return ISG_OK;
}

int isg_sweep_test_stall(isg_sim* h) {
    if (!h) { set_error("isg_sweep_test_stall: NULL handle"); return ISG_ERR_ARG; }
    if (!sweeps_in_one_launch(h, 64)) {
        set_error("isg_sweep_test_stall: this handle's sweeps do not run as multi-pass launches");
        return ISG_ERR_STATE;
    }
    h->stall_next = true;
    return ISG_OK;
}

int isg_sweeps_done(const isg_sim* h, int64_t* n) {
    if (!h || !n) { set_error("isg_sweeps_done: NULL argument"); return ISG_ERR_ARG; }
    *n = h->sweeps;
    return ISG_OK;
}

int isg_energy(isg_sim* h, int64_t* E, void* stream) {
    if (!h || !E) { set_error("isg_energy: NULL argument"); return ISG_ERR_ARG; }
    return energy_sync(h, E, (cudaStream_t)stream);
}

int isg_tracked_energy(isg_sim* h, int64_t* E) {
    if (!h || !E) { set_error("isg_tracked_energy: NULL argument"); return ISG_ERR_ARG; }
    long long w[6] = {0, 0, 0, 0, 0, 0};  // scal[0..5]: dE, ..., the error word
    cudaError_t e = cudaMemcpyAsync(w, h->scal, sizeof w, cudaMemcpyDeviceToHost, h->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "isg_tracked_energy");
    if (const int rc = wait_error(h, w[5], h->last_stream)) return rc;
    *E = h->E0 + (int64_t)w[0];
    return ISG_OK;
}

int isg_overlap(const isg_sim* a, const isg_sim* b, int64_t* Q, void* stream) {
    if (!a || !b || !Q) { set_error("isg_overlap: NULL argument"); return ISG_ERR_ARG; }
    if (a->L != b->L || a->seed_J != b->seed_J) {
        set_error("isg_overlap: handles differ in L or seed_J");
        return ISG_ERR_MISMATCH;
    }
    cudaStream_t s = (cudaStream_t)stream;
    long long* acc = a->scal + 1;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(long long), s);
    if (e == cudaSuccess) e = launch_overlap(a, b, acc, s);
    long long nd = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nd, acc, sizeof nd, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "isg_overlap");
    *Q = (int64_t)a->L * a->L * a->L - 2 * (int64_t)nd;
    return ISG_OK;
}

int isg_hash(const isg_sim* h, uint64_t* H, void* stream) {
    if (!h || !H) { set_error("isg_hash: NULL argument"); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* acc = (unsigned long long*)(h->scal + 2);
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_hash(h, acc, s);
    unsigned long long v = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, acc, sizeof v, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "isg_hash");
    *H = (uint64_t)v;
    return ISG_OK;
}

// Host <-> device transfer of an int8 array through a temporary device buffer.
static int read_int8(const isg_sim* hc, int8_t* out, size_t n, size_t need, cudaStream_t s, bool couplings) {
    isg_sim* h = const_cast<isg_sim*>(hc);
    if (n < need) { set_error("read: buffer holds %zu values, %zu needed", n, need); return ISG_ERR_ARG; }
    int8_t* d = (int8_t*)dev_alloc(h, need);
    if (!d) { set_error("read: device allocation failed"); return ISG_ERR_NOMEM; }
    cudaError_t e = couplings ? launch_unpack_couplings(h, d, s) : launch_unpack_spins_fast(h, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, need, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(h, d);
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "read");
}

// Spins from int8 +-1: validated and packed in one pass into a scratch copy of
// the two spin planes, which replaces them only if every value was +1 or -1.
static int write_spins_int8(isg_sim* h, const int8_t* in, size_t n, size_t need, cudaStream_t s) {
    if (n < need) { set_error("write: buffer holds %zu values, %zu needed", n, need); return ISG_ERR_ARG; }
    int8_t* d = (int8_t*)dev_alloc(h, need);
    unsigned char* scratch = (unsigned char*)dev_alloc(h, 2 * (size_t)h->plane_bytes);
    int* bad = (int*)dev_alloc(h, sizeof(int));
    if (!d || !scratch || !bad) {
        dev_free(h, d);
        dev_free(h, scratch);
        dev_free(h, bad);
        set_error("write: device allocation failed");
        return ISG_ERR_NOMEM;
    }
    int hbad = 0;
    cudaError_t e = cudaMemcpyAsync(d, in, need, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_pack_spins_checked(h, d, scratch, bad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int c = 0; c < 2 && e == cudaSuccess && !hbad; ++c)
        e = cudaMemcpyAsync(h->plane(c, 0), scratch + (size_t)c * h->plane_bytes, (size_t)h->plane_bytes,
                            cudaMemcpyDeviceToDevice, s);
    dev_free(h, d);
    dev_free(h, scratch);
    dev_free(h, bad);
    if (e != cudaSuccess) return cuda_fail(e, "write");
    if (hbad) { set_error("write: values must be +1 or -1"); return ISG_ERR_ARG; }
    return restart_tracking(h, s);
}

static int write_int8(isg_sim* h, const int8_t* in, size_t n, size_t need, cudaStream_t s, bool couplings) {
    if (!couplings) return write_spins_int8(h, in, n, need, s);
    if (n < need) { set_error("write: buffer holds %zu values, %zu needed", n, need); return ISG_ERR_ARG; }
    int8_t* d = (int8_t*)dev_alloc(h, need);
    int* bad = (int*)dev_alloc(h, sizeof(int));
    if (!d || !bad) {
        dev_free(h, d);
        dev_free(h, bad);
        set_error("write: device allocation failed");
        return ISG_ERR_NOMEM;
    }
    int hbad = 0;
    cudaError_t e = cudaMemcpyAsync(d, in, need, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_check_pm1(d, (int64_t)need, bad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && !hbad) {
        e = launch_pack_couplings(h, d, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    dev_free(h, d);
    dev_free(h, bad);
    if (e != cudaSuccess) return cuda_fail(e, "write");
    if (hbad) { set_error("write: values must be +1 or -1"); return ISG_ERR_ARG; }
    return restart_tracking(h, s);
}

int isg_read_spins(const isg_sim* h, int8_t* out, size_t n, void* stream) {
    if (!h || !out) { set_error("isg_read_spins: NULL argument"); return ISG_ERR_ARG; }
    return read_int8(h, out, n, (size_t)h->L * h->L * h->L, (cudaStream_t)stream, false);
}

int isg_write_spins(isg_sim* h, const int8_t* in, size_t n, void* stream) {
    if (!h || !in) { set_error("isg_write_spins: NULL argument"); return ISG_ERR_ARG; }
    return write_int8(h, in, n, (size_t)h->L * h->L * h->L, (cudaStream_t)stream, false);
}

int isg_read_spins_packed(const isg_sim* hc, uint8_t* out, size_t nbytes, void* stream) {
    if (!hc || !out) { set_error("isg_read_spins_packed: NULL argument"); return ISG_ERR_ARG; }
    isg_sim* h = const_cast<isg_sim*>(hc);
    const int64_t N = (int64_t)h->L * h->L * h->L;
    const size_t need = (size_t)((N + 7) / 8);
    if (nbytes < need) { set_error("isg_read_spins_packed: buffer holds %zu bytes, %zu needed", nbytes, need); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* d = (uint32_t*)dev_alloc(h, (size_t)((N + 31) / 32) * 4);
    if (!d) { set_error("isg_read_spins_packed: device allocation failed"); return ISG_ERR_NOMEM; }
    cudaError_t e = launch_unpack_spins_bits(h, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, need, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(h, d);
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "isg_read_spins_packed");
}

int isg_exchange_async(isg_sim* h, const uint8_t* in, uint8_t* out, size_t nbytes, int64_t sweeps, long long* E_out,
                       void* stream) {
    if (!h || sweeps < 0) { set_error("isg_exchange_async: bad handle or sweeps"); return ISG_ERR_ARG; }
    const int64_t N = (int64_t)h->L * h->L * h->L;
    const size_t need = (size_t)((N + 7) / 8);
    if ((in || out) && nbytes < need) {
        set_error("isg_exchange_async: buffers hold %zu bytes, %zu needed", nbytes, need);
        return ISG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((in || out) && !h->stage) {
        h->stage = (uint32_t*)dev_alloc(h, (size_t)((N + 31) / 32) * 4);
        if (!h->stage) { set_error("isg_exchange_async: device allocation failed"); return ISG_ERR_NOMEM; }
    }
    cudaError_t e = cudaSuccess;
    int64_t left = sweeps;
    if (in) {
        e = cudaMemcpyAsync(h->stage, in, need, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_pack_spins_bits(h, h->stage, s);
        if (e == cudaSuccess && sweeps > 0) {
            // the first red pass counts the new configuration's bonds before its
            // flips, so no separate energy pass over the planes is needed
            e = cudaMemsetAsync(h->scal, 0, 2 * sizeof(long long), s);
            if (e == cudaSuccess) e = launch_flip_fast(h, 0, s, (unsigned long long*)(h->scal + 1));
            if (e == cudaSuccess) {
                restart_after_pass_kernel<<<1, 1, 0, s>>>(h->scal, 3 * (long long)N, (long long)h->E0);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = launch_flip_fast(h, 1, s);
            if (e == cudaSuccess) {
                h->sweeps += 1;
                left -= 1;
            }
        } else if (e == cudaSuccess) {
            e = cudaMemsetAsync(h->scal + 1, 0, sizeof(long long), s);
            if (e == cudaSuccess) e = launch_energy(h, h->scal + 1, s);
            if (e == cudaSuccess) {
                restart_on_device_kernel<<<1, 1, 0, s>>>(h->scal, 3 * (long long)N, (long long)h->E0);
                e = cudaGetLastError();
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "isg_exchange_async: spins in");
    }
    h->last_stream = s;
    if (left > 0) {
        const int rc = isg_sweep(h, left, stream);
        if (rc) return rc;
    }
    if (out) {
        e = launch_unpack_spins_bits(h, h->stage, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->stage, need, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "isg_exchange_async: spins out");
    }
    if (E_out) {
        tracked_word_kernel<<<1, 1, 0, s>>>(h->scal, (long long)h->E0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(E_out, h->scal + 4, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "isg_exchange_async: energy out");
    }
    return ISG_OK;
}

int isg_write_spins_packed(isg_sim* h, const uint8_t* in, size_t nbytes, void* stream) {
    if (!h || !in) { set_error("isg_write_spins_packed: NULL argument"); return ISG_ERR_ARG; }
    const int64_t N = (int64_t)h->L * h->L * h->L;
    const size_t need = (size_t)((N + 7) / 8);
    if (nbytes < need) { set_error("isg_write_spins_packed: buffer holds %zu bytes, %zu needed", nbytes, need); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* d = (uint32_t*)dev_alloc(h, (size_t)((N + 31) / 32) * 4);
    if (!d) { set_error("isg_write_spins_packed: device allocation failed"); return ISG_ERR_NOMEM; }
    cudaError_t e = cudaMemcpyAsync(d, in, need, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_pack_spins_bits(h, d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(h, d);
    if (e != cudaSuccess) return cuda_fail(e, "isg_write_spins_packed");
    return restart_tracking(h, s);
}

int isg_read_couplings(const isg_sim* h, int8_t* out, size_t n, void* stream) {
    if (!h || !out) { set_error("isg_read_couplings: NULL argument"); return ISG_ERR_ARG; }
    return read_int8(h, out, n, 3 * (size_t)h->L * h->L * h->L, (cudaStream_t)stream, true);
}

int isg_write_couplings(isg_sim* h, const int8_t* in, size_t n, void* stream) {
    if (!h || !in) { set_error("isg_write_couplings: NULL argument"); return ISG_ERR_ARG; }
    return write_int8(h, in, n, 3 * (size_t)h->L * h->L * h->L, (cudaStream_t)stream, true);
}

// ---------------------------------------------------------------- checkpoint
struct SaveHeader {
    char magic[8];
    uint32_t version, L, kind, wbits;
    double beta;
    uint64_t seed_J, seed_spin, seed_rng;
    int64_t R, S, sweeps, E0, dE, plane_bytes, rng_words;
};

static const char kMagic[8] = {'I', 'S', 'G', 'C', 'K', 'P', 'T', '2'};

int isg_save(const isg_sim* h, void* buf, size_t* n, void* stream) {
    if (!h || !n) { set_error("isg_save: NULL argument"); return ISG_ERR_ARG; }
    const size_t rng_words = (size_t)h->S * rng_state_words(h->kind);
    const size_t need = sizeof(SaveHeader) + (size_t)h->plane_bytes * 8 + rng_words * 4 + (size_t)h->S * 4;
    if (!buf) { *n = need; return ISG_OK; }
    if (*n < need) { *n = need; set_error("isg_save: buffer too small"); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    SaveHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, kMagic, 8);
    hd.version = 1;
    hd.L = (uint32_t)h->L;
    hd.kind = (uint32_t)h->kind;
    hd.wbits = (uint32_t)h->wbits;
    hd.beta = h->beta;
    hd.seed_J = h->seed_J;
    hd.seed_spin = h->seed_spin;
    hd.seed_rng = h->seed_rng;
    hd.R = h->R;
    hd.S = h->S;
    hd.sweeps = h->sweeps;
    hd.E0 = h->E0;
    hd.plane_bytes = h->plane_bytes;
    hd.rng_words = (int64_t)rng_words;
    long long d = 0;
    unsigned char* p = (unsigned char*)buf + sizeof hd;
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&d, h->scal, sizeof d, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->planes, (size_t)h->plane_bytes * 8, cudaMemcpyDeviceToHost, s);
    p += (size_t)h->plane_bytes * 8;
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->rng, rng_words * 4, cudaMemcpyDeviceToHost, s);
    p += rng_words * 4;
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->rng_pos, (size_t)h->S * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "isg_save");
    hd.dE = d;
    memcpy(buf, &hd, sizeof hd);
    *n = need;
    return ISG_OK;
}

int isg_load(const void* buf, size_t n, isg_sim** out) {
    if (!buf || !out) { set_error("isg_load: NULL argument"); return ISG_ERR_ARG; }
    *out = nullptr;
    SaveHeader hd;
    if (n < sizeof hd) { set_error("isg_load: truncated buffer"); return ISG_ERR_ARG; }
    memcpy(&hd, buf, sizeof hd);
    if (memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1) { set_error("isg_load: not a checkpoint"); return ISG_ERR_ARG; }
    if (hd.L < 4 || hd.L > 2048 || (hd.L & 1) || !rng_kind_valid((int)hd.kind) || !beta_ok(hd.beta)) {
        set_error("isg_load: corrupt header");
        return ISG_ERR_ARG;
    }
    isg_sim* h = new_sim();
    if (!h) { set_error("isg_load: out of host memory"); return ISG_ERR_NOMEM; }
    h->L = (int)hd.L;
    h->kind = (int)hd.kind;
    h->beta = hd.beta;
    h->seed_J = hd.seed_J;
    h->seed_spin = hd.seed_spin;
    h->seed_rng = hd.seed_rng;
    {
        // 64-bit words where 32-bit ones would be chosen: the saved handle was a batch member
        const int half = h->L / 2, w64 = (half + 63) / 64, w32 = (half + 31) / 32;
        h->member = hd.wbits == 64 && 2 * w64 != w32;
    }
    thresholds(h->beta, h->thr);
    int rc = alloc_sim(h);
    if (rc) { free_sim(h); return rc; }
    const size_t rng_words = (size_t)h->S * rng_state_words(h->kind);
    const size_t need = sizeof hd + (size_t)h->plane_bytes * 8 + rng_words * 4 + (size_t)h->S * 4;
    if (n < need || hd.plane_bytes != h->plane_bytes || hd.S != h->S || hd.R != h->R ||
        hd.rng_words != (int64_t)rng_words || (int)hd.wbits != h->wbits) {
        free_sim(h);
        set_error("isg_load: buffer does not match its header");
        return ISG_ERR_ARG;
    }
    const unsigned char* p = (const unsigned char*)buf + sizeof hd;
    long long d = hd.dE;
    cudaError_t e = cudaMemcpy(h->planes, p, (size_t)h->plane_bytes * 8, cudaMemcpyHostToDevice);
    p += (size_t)h->plane_bytes * 8;
    if (e == cudaSuccess) e = cudaMemcpy(h->rng, p, rng_words * 4, cudaMemcpyHostToDevice);
    p += rng_words * 4;
    if (e == cudaSuccess) e = cudaMemcpy(h->rng_pos, p, (size_t)h->S * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->scal, &d, sizeof d, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_sim(h); return cuda_fail(e, "isg_load"); }
    h->sweeps = hd.sweeps;
    h->E0 = hd.E0;
    *out = h;
    return ISG_OK;
}

// ------------------------------------------------------------------ testing
int isg_stencil_decisions(const uint16_t* code, const uint32_t* draw, int64_t n, const uint32_t thr[3],
                          uint8_t* flip, uint8_t* u) {
    if (!code || !draw || !thr || !flip || !u || n < 0) { set_error("isg_stencil_decisions: bad argument"); return ISG_ERR_ARG; }
    if (n == 0) return ISG_OK;
    uint16_t* dc = nullptr;
    uint32_t* dd = nullptr;
    uint8_t *df = nullptr, *du = nullptr;
    cudaError_t e = cudaMalloc(&dc, n * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dd, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&df, n);
    if (e == cudaSuccess) e = cudaMalloc(&du, n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, code, n * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dd, draw, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_stencil(dc, dd, n, thr[0], thr[1], thr[2], df, du, 0);
    if (e == cudaSuccess) e = cudaMemcpy(flip, df, n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(u, du, n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dd);
    cudaFree(df);
    cudaFree(du);
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "isg_stencil_decisions");
}

int isg_peek_draws(const isg_sim* h, int64_t t, int64_t n, uint32_t* out) {
    if (!h || !out || t < 0 || t >= h->S || n < 0) { set_error("isg_peek_draws: bad argument"); return ISG_ERR_ARG; }
    if (n == 0) return ISG_OK;
    isg_sim* hm = const_cast<isg_sim*>(h);
    uint32_t* d = (uint32_t*)dev_alloc(hm, (size_t)n * 4);
    if (!d) { set_error("isg_peek_draws: allocation failed"); return ISG_ERR_NOMEM; }
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    if (e == cudaSuccess) e = launch_peek_draws(h, t, n, d, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)n * 4, cudaMemcpyDeviceToHost);
    dev_free(hm, d);
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "isg_peek_draws");
}

}  // extern "C"
