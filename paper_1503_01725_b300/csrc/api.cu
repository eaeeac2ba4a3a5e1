// api.cu -- the extern "C" entry points of liblsm.so (declared in include/lsm.h).
#include <atomic>
#include <math.h>
#include <mutex>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "handles.cuh"

namespace lsm {

lsm_status model_create(const lsm_psr_model *, lsm_model **);
lsm_status read_fallbacks(int64_t *, int);
extern int g_stage_polls;
namespace dn {
extern unsigned long long g_conv_wait_ns;
}
void model_destroy(lsm_model *);
lsm_status model_commission(const lsm_model *, const double *, int32_t, lsm_model **);
lsm_status model_weights(const lsm_model *, double *);
lsm_status build_psl(const lsm_model *, const lsm_beams *, int64_t, const int64_t *, lsm_psl **, cudaStream_t,
                     bool);
lsm_status free_psl(lsm_psl *);
lsm_status resolve_psl(lsm_psl *);
lsm_status create_phantom(const lsm_phantom_desc *, lsm_phantom **, cudaStream_t, bool);
void free_phantom(lsm_phantom *);
lsm_status sample_public(const lsm_psl *, uint64_t, uint64_t, int64_t, double, const lsm_particles *, cudaStream_t);
lsm_status transport_particles(const lsm_phantom *, const lsm_particles *, int64_t, uint64_t, lsm_tally *,
                               const lsm_run_opts *, cudaStream_t);
lsm_status run_plan(const lsm_psl *, const lsm_phantom *, lsm_tally *, uint64_t, const lsm_run_opts *, cudaStream_t);
lsm_status fold_batch(lsm_tally *, cudaStream_t, bool);
lsm_status flush_partials(lsm_tally *, cudaStream_t);
lsm_status dose_impl(const lsm_tally *, const lsm_phantom *, double, double *, double *, lsm_mem, cudaStream_t);
lsm_status basis_impl(const lsm_tally *, const lsm_psl *, const lsm_phantom *, const uint16_t *, lsm_mem, double *,
                      lsm_mem, cudaStream_t, bool);
lsm_status commission(const double *, int32_t, int32_t, const double *, lsm_mem, const lsm_nnls_opts *, double *,
                      lsm_nnls_report *, cudaStream_t);

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

// ---- event timers ----
struct TimerRec {
    int which;
    cudaEvent_t a, b;
    long long launches;   // kernels launched between the two events
};
static std::mutex g_tm;
static bool g_timing = false;
static std::vector<TimerRec> g_open;      // recorded, not yet resolved
static std::vector<cudaEvent_t> g_pool;
static double g_ms[LSM_N_TIMERS];
static long long g_cnt[LSM_N_TIMERS];
static thread_local long long g_cur_launch0 = 0;

static cudaEvent_t ev_get()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

static void record(cudaEvent_t e, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}

int timer_begin(int which, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_tm);
    if (!g_timing) return -1;
    TimerRec r;
    r.which = which;
    r.a = ev_get();
    r.b = ev_get();
    r.launches = 0;
    record(r.a, st);
    g_open.push_back(r);
    g_cur_launch0 = g_launches.load();
    return (int)g_open.size() - 1;
}

void timer_end(int token, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_tm);
    if (token < 0 || token >= (int)g_open.size()) return;
    record(g_open[token].b, st);
    g_open[token].launches = g_launches.load() - g_cur_launch0;
}

// Timers recorded while a stream is captured become event nodes of the graph;
// they are detached from the open list and resolved after every replay.
size_t timer_mark()
{
    std::lock_guard<std::mutex> lk(g_tm);
    return g_open.size();
}

void *timer_detach(size_t from)
{
    std::lock_guard<std::mutex> lk(g_tm);
    if (from >= g_open.size()) return nullptr;
    auto *v = new std::vector<TimerRec>(g_open.begin() + from, g_open.end());
    g_open.resize(from);
    return v;
}

void timer_replayed(void *set)
{   // the replay's events have completed (the caller synchronised)
    if (!set) return;
    std::lock_guard<std::mutex> lk(g_tm);
    for (const TimerRec &r : *(std::vector<TimerRec> *)set) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) g_ms[r.which] += t;
        g_cnt[r.which] += r.launches;
    }
}

void timer_free(void *set)
{
    if (!set) return;
    std::lock_guard<std::mutex> lk(g_tm);
    for (const TimerRec &r : *(std::vector<TimerRec> *)set) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    delete (std::vector<TimerRec> *)set;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t next_uid()
{
    static std::atomic<unsigned long long> n{0};
    return (uint64_t)n.fetch_add(1, std::memory_order_relaxed) + 1;
}
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool timing_enabled()
{
    std::lock_guard<std::mutex> lk(g_tm);
    return g_timing;
}

lsm_status set_cuda_error(cudaError_t e, const char *where)
{
    snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
    return LSM_ERR_CUDA;
}

lsm_status set_arg_error(const char *msg)
{
    snprintf(g_err, sizeof(g_err), "%s", msg);
    return LSM_ERR_ARG;
}

cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t st)
{
    // keep up to 64 GiB of freed blocks in the pool of each device that allocates
    static std::mutex m;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(m);
        if (!done[dev]) {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = 64ull << 30;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            done[dev] = true;
        }
    }
    return cudaMallocAsync(p, bytes, st);
}

void dev_free(void *p)
{
    if (p) cudaFreeAsync(p, 0);
}

lsm_status set_io_error(const char *what, const char *path, int err)
{
    snprintf(g_err, sizeof(g_err), "%s %s: %s", what, path ? path : "(null)", err ? strerror(err) : "short transfer");
    return LSM_ERR_IO;
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

}  // namespace lsm

using namespace lsm;

static cudaStream_t S(lsm_stream s) { return (cudaStream_t)s; }

extern "C" {

const char *lsm_last_error(void) { return lsm::g_err; }

lsm_status lsm_timing_enable(int on)
{
    std::lock_guard<std::mutex> lk(lsm::g_tm);
    lsm::g_timing = on != 0;
    return LSM_OK;
}

lsm_status lsm_timing_read(double ms[LSM_N_TIMERS], int64_t launches[LSM_N_TIMERS], int reset)
{
    LSM_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(lsm::g_tm);
    for (auto &r : lsm::g_open) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) lsm::g_ms[r.which] += t;
        lsm::g_cnt[r.which] += r.launches;
        lsm::g_pool.push_back(r.a);
        lsm::g_pool.push_back(r.b);
    }
    lsm::g_open.clear();
    for (int i = 0; i < LSM_N_TIMERS; ++i) {
        if (ms) ms[i] = lsm::g_ms[i];
        if (launches) launches[i] = lsm::g_cnt[i];
        if (reset) { lsm::g_ms[i] = 0.0; lsm::g_cnt[i] = 0; }
    }
    return LSM_OK;
}

int64_t lsm_launch_count(void) { return (int64_t)lsm::g_launches.load(); }

lsm_status lsm_set_wait_limits(int64_t stage_polls, int64_t conv_wait_ns)
{
    if (stage_polls > (1ll << 30)) return set_arg_error("lsm_set_wait_limits: stage_polls <= 2^30");
    if (stage_polls >= 0) lsm::g_stage_polls = (int)stage_polls;
    if (conv_wait_ns >= 0) lsm::dn::g_conv_wait_ns = (unsigned long long)conv_wait_ns;
    return LSM_OK;
}

lsm_status lsm_run_fallbacks(int64_t *count, int reset) { return read_fallbacks(count, reset); }

lsm_status lsm_model_create(const lsm_psr_model *psr, lsm_model **out) { return model_create(psr, out); }

void lsm_model_destroy(lsm_model *model) { model_destroy(model); }

lsm_status lsm_build_psl(const lsm_model *model, const lsm_beams *beams, int64_t n_hist,
                         const int64_t *per_psr_hist, lsm_psl **out, lsm_stream stream)
{
    const int tk = timer_begin(0, S(stream));
    lsm_status rc = build_psl(model, beams, n_hist, per_psr_hist, out, S(stream), false);
    timer_end(tk, S(stream));
    return rc;
}

lsm_status lsm_build_psl_async(const lsm_model *model, const lsm_beams *beams, int64_t n_hist,
                               const int64_t *per_psr_hist, lsm_psl **out, lsm_stream stream)
{
    const int tk = timer_begin(0, S(stream));
    lsm_status rc = build_psl(model, beams, n_hist, per_psr_hist, out, S(stream), true);
    timer_end(tk, S(stream));
    return rc;
}

void lsm_psl_destroy(lsm_psl *psl) { free_psl(psl); }

lsm_status lsm_psl_info(const lsm_psl *P, int64_t info[4], double *denom)
{
    if (!P || !info) return set_arg_error("lsm_psl_info: NULL argument");
    lsm_status r = resolve_psl(const_cast<lsm_psl *>(P));
    if (r) return r;
    info[0] = P->n_xy; info[1] = P->n_ent; info[2] = P->plan_size; info[3] = P->per_psr;
    if (denom) *denom = P->denom;
    return LSM_OK;
}

lsm_status lsm_psl_copy(const lsm_psl *P, int which, void *dst)
{
    if (!P || !dst) return set_arg_error("lsm_psl_copy: NULL argument");
    lsm_status r = resolve_psl(const_cast<lsm_psl *>(P));
    if (r) return r;
    const size_t npsl = (size_t)P->n_xy * P->n_xy;
    LSM_CUDA(cudaDeviceSynchronize());
    switch (which) {
    case 0: LSM_CUDA(cudaMemcpy(dst, P->d_wpsl, 3 * (size_t)P->n_e * npsl * 8, cudaMemcpyDeviceToHost)); break;
    case 1: LSM_CUDA(cudaMemcpy(dst, P->d_incl, (size_t)P->n_beams * 2 * npsl, cudaMemcpyDeviceToHost)); break;
    case 2: LSM_CUDA(cudaMemcpy(dst, P->d_area, (size_t)P->n_beams * 64, cudaMemcpyDeviceToHost)); break;
    case 3: LSM_CUDA(cudaMemcpy(dst, P->d_count, (size_t)P->ncell * 8, cudaMemcpyDeviceToHost)); break;
    case 4: LSM_CUDA(cudaMemcpy(dst, P->d_start, (size_t)(P->n_ent + 1) * 8, cudaMemcpyDeviceToHost)); break;
    case 5: {
        EntryRec *h = (EntryRec *)malloc((size_t)P->n_ent * sizeof(EntryRec));
        cudaError_t e = cudaMemcpy(h, P->d_ent, (size_t)P->n_ent * sizeof(EntryRec), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { free(h); return set_cuda_error(e, "lsm_psl_copy"); }
        int32_t *o = (int32_t *)dst;
        for (int64_t k = 0; k < P->n_ent; ++k) {
            o[6 * k + 0] = h[k].beam; o[6 * k + 1] = h[k].stype; o[6 * k + 2] = h[k].ebin;
            o[6 * k + 3] = h[k].ix; o[6 * k + 4] = h[k].iy;
            o[6 * k + 5] = P->per_psr ? ((h[k].stype * P->n_e + h[k].ebin) * P->n_r + h[k].fixed_ring) : -1;
        }
        free(h);
        break;
    }
    case 6: LSM_CUDA(cudaMemcpy(dst, P->d_escale, (size_t)P->n_ent * 8, cudaMemcpyDeviceToHost)); break;
    default: return set_arg_error("lsm_psl_copy: unknown table");
    }
    return LSM_OK;
}

lsm_status lsm_sample(const lsm_psl *psl, uint64_t seed, uint64_t hist_begin, int64_t n, double z_surface,
                      const lsm_particles *out, lsm_stream stream)
{
    return sample_public(psl, seed, hist_begin, n, z_surface, out, S(stream));
}

lsm_status lsm_phantom_create(const lsm_phantom_desc *desc, lsm_phantom **out, lsm_stream stream)
{
    const int tk = timer_begin(7, S(stream));
    lsm_status rc = create_phantom(desc, out, S(stream), false);
    timer_end(tk, S(stream));
    return rc;
}

lsm_status lsm_phantom_create_async(const lsm_phantom_desc *desc, lsm_phantom **out, lsm_stream stream)
{
    const int tk = timer_begin(7, S(stream));
    lsm_status rc = create_phantom(desc, out, S(stream), true);
    timer_end(tk, S(stream));
    return rc;
}

lsm_status lsm_phantom_check(const lsm_phantom *ph, lsm_stream stream)
{
    if (!ph) return set_arg_error("lsm_phantom_check: NULL phantom");
    unsigned bad = 0;
    LSM_CUDA(cudaMemcpyAsync(&bad, ph->d_flags + 2, 4, cudaMemcpyDeviceToHost, S(stream)));
    LSM_CUDA(cudaStreamSynchronize(S(stream)));
    if (bad) return set_arg_error("lsm_phantom_check: densities must be in [1e-4, 25] and materials in {0, 1}");
    return LSM_OK;
}

void lsm_phantom_destroy(lsm_phantom *ph) { free_phantom(ph); }

lsm_status lsm_phantom_tables(const lsm_phantom *ph, float *out, double grid[2])
{
    if (!ph || !out) return set_arg_error("lsm_phantom_tables: NULL argument");
    LSM_CUDA(cudaDeviceSynchronize());
    LSM_CUDA(cudaMemcpy(out, ph->d_xs, 2 * kGrid * sizeof(float4), cudaMemcpyDeviceToHost));
    LSM_CUDA(cudaMemcpy(out + 8 * kGrid, ph->d_mumax, kGrid * 4 + kKnE * kKnU * 4, cudaMemcpyDeviceToHost));
    if (grid) { grid[0] = kLnEmin; grid[1] = (kLnEmax - kLnEmin) / (kGrid - 1); }
    return LSM_OK;
}

lsm_status lsm_tally_create(const lsm_phantom *ph, const lsm_tally_desc *d, lsm_tally **out, lsm_stream stream)
{
    if (!ph || !d || !out) return set_arg_error("lsm_tally_create: NULL argument");
    *out = nullptr;
    const int64_t nvox = (int64_t)ph->nx * ph->ny * ph->nz;
    int64_t ncell = nvox;
    if (d->mode == 1) {
        if (!d->idx3d || d->n_rows < 1 || d->n_rows > 65535 || d->n_psr < 1 || d->n_psr > 65535 || d->n_beams < 1 ||
            d->n_beams > 16)
            return set_arg_error("lsm_tally_create: basis tally needs idx3d, 1..65535 rows and PSRs, 1..16 beams");
        ncell = (int64_t)d->n_beams * d->n_rows * d->n_psr;
    } else if (d->mode != 0) {
        return set_arg_error("lsm_tally_create: mode must be 0 or 1");
    }
    lsm_tally *t = (lsm_tally *)calloc(1, sizeof(lsm_tally));
    cudaGetDevice(&t->device);
    t->mode = d->mode; t->n_rows = d->n_rows; t->n_psr = d->n_psr; t->n_beams = d->n_beams;
    t->ncell = ncell; t->nvox = nvox;
    t->part_slots = 1;
    cudaStream_t st = S(stream);
    cudaError_t e = cudaSuccess;
    do {
        if ((e = dev_malloc((void **)&t->d_part, (size_t)ncell * 4 + 16, st)) != cudaSuccess) break;
        if ((e = dev_malloc((void **)&t->d_batch, (size_t)ncell * 8 + 16, st)) != cudaSuccess) break;
        if ((e = dev_malloc((void **)&t->d_s1, (size_t)ncell * 8 + 16, st)) != cudaSuccess) break;
        if ((e = dev_malloc((void **)&t->d_s2, (size_t)ncell * 8 + 16, st)) != cudaSuccess) break;
        if ((e = dev_malloc((void **)&t->d_stats, sizeof(RunStats), st)) != cudaSuccess) break;
        if (d->mode == 1) {
            if ((e = dev_malloc((void **)&t->d_idx, (size_t)nvox * 2, st)) != cudaSuccess) break;
            e = cudaMemcpyAsync(t->d_idx, d->idx3d, (size_t)nvox * 2,
                                d->idx3d_mem == LSM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) break;
            // a host array is read before returning, also when it is pinned
            // (a copy from pinned memory would otherwise run later)
            if (d->idx3d_mem == LSM_MEM_HOST && (e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        }
        if ((e = cudaMemsetAsync(t->d_part, 0, (size_t)ncell * 4, st)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(t->d_batch, 0, (size_t)ncell * 8, st)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(t->d_s1, 0, (size_t)ncell * 8, st)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(t->d_s2, 0, (size_t)ncell * 8, st)) != cudaSuccess) break;
        e = cudaMemsetAsync(t->d_stats, 0, sizeof(RunStats), st);
    } while (0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        dev_free(t->d_part); dev_free(t->d_batch); dev_free(t->d_s1); dev_free(t->d_s2); dev_free(t->d_stats);
        dev_free(t->d_idx);
        free(t);
        return set_cuda_error(e, "lsm_tally_create");
    }
    // row indices must stay inside n_rows (checked once, on the host copy when available)
    if (d->mode == 1 && d->idx3d_mem == LSM_MEM_HOST) {
        for (int64_t i = 0; i < nvox; ++i)
            if (d->idx3d[i] > d->n_rows) {
                lsm_tally_destroy(t);
                return set_arg_error("lsm_tally_create: idx3d holds a row beyond n_rows");
            }
    }
    *out = t;
    return LSM_OK;
}

// The tally's memory returns to the pool in the order of the legacy default
// stream; its own graph stream is drained first.
void lsm_tally_destroy(lsm_tally *t)
{
    if (!t) return;
    if (t->gstream) cudaStreamSynchronize((cudaStream_t)t->gstream);
    if (t->pstream) cudaStreamSynchronize((cudaStream_t)t->pstream);
    dev_free(t->d_part); dev_free(t->d_batch); dev_free(t->d_s1); dev_free(t->d_s2); dev_free(t->d_stats);
    dev_free(t->d_idx);
    dev_free(t->ws);
    dev_free(t->ws2);
    if (t->pstream) {
        cudaStreamDestroy((cudaStream_t)t->pstream);
        cudaEventDestroy((cudaEvent_t)t->pev[0]);
        cudaEventDestroy((cudaEvent_t)t->pev[1]);
    }
    if (t->gexec) cudaGraphExecDestroy((cudaGraphExec_t)t->gexec);
    timer_free(t->gtimers);
    if (t->gstream) {
        cudaStreamDestroy((cudaStream_t)t->gstream);
        cudaEventDestroy((cudaEvent_t)t->gev[0]);
        cudaEventDestroy((cudaEvent_t)t->gev[1]);
    }
    free(t);
}

lsm_status lsm_tally_reset(lsm_tally *t, lsm_stream stream)
{
    if (!t) return set_arg_error("lsm_tally_reset: NULL tally");
    cudaStream_t st = S(stream);
    LSM_CUDA(cudaMemsetAsync(t->d_part, 0, (size_t)t->part_slots * t->ncell * 4, st));
    LSM_CUDA(cudaMemsetAsync(t->d_batch, 0, (size_t)t->ncell * 8, st));
    LSM_CUDA(cudaMemsetAsync(t->d_s1, 0, (size_t)t->ncell * 8, st));
    LSM_CUDA(cudaMemsetAsync(t->d_s2, 0, (size_t)t->ncell * 8, st));
    LSM_CUDA(cudaMemsetAsync(t->d_stats, 0, sizeof(RunStats), st));
    t->n_batches = 0;
    return LSM_OK;
}

lsm_status lsm_tally_end_batch(lsm_tally *t, lsm_stream stream)
{
    if (!t) return set_arg_error("lsm_tally_end_batch: NULL tally");
    lsm_status rc = flush_partials(t, S(stream));
    if (rc) return rc;
    return fold_batch(t, S(stream), true);
}

lsm_status lsm_tally_read(lsm_tally *t, double *s1, double *s2, lsm_mem mem, int32_t *n_batches, lsm_stream stream)
{
    if (!t) return set_arg_error("lsm_tally_read: NULL tally");
    cudaStream_t st = S(stream);
    const cudaMemcpyKind k = mem == LSM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (s1) LSM_CUDA(cudaMemcpyAsync(s1, t->d_s1, (size_t)t->ncell * 8, k, st));
    if (s2) LSM_CUDA(cudaMemcpyAsync(s2, t->d_s2, (size_t)t->ncell * 8, k, st));
    if (mem == LSM_MEM_HOST) LSM_CUDA(cudaStreamSynchronize(st));
    if (n_batches) *n_batches = t->n_batches;
    return LSM_OK;
}

lsm_status lsm_tally_load(lsm_tally *t, const double *s1, const double *s2, int32_t n_batches,
                          const double ledger[4], const int64_t stats[11], lsm_mem mem, lsm_stream stream)
{
    if (!t || !s1 || !s2) return set_arg_error("lsm_tally_load: NULL argument");
    if (n_batches < 0) return set_arg_error("lsm_tally_load: n_batches < 0");
    cudaStream_t st = S(stream);
    const cudaMemcpyKind k = mem == LSM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    LSM_CUDA(cudaMemcpyAsync(t->d_s1, s1, (size_t)t->ncell * 8, k, st));
    LSM_CUDA(cudaMemcpyAsync(t->d_s2, s2, (size_t)t->ncell * 8, k, st));
    LSM_CUDA(cudaMemsetAsync(t->d_part, 0, (size_t)t->part_slots * t->ncell * 4, st));
    LSM_CUDA(cudaMemsetAsync(t->d_batch, 0, (size_t)t->ncell * 8, st));
    RunStats h;
    memset(&h, 0, sizeof(h));
    if (ledger) for (int i = 0; i < 4; ++i) h.ledger[i] = ledger[i];
    if (stats) for (int i = 0; i < 11; ++i) h.c[i] = (unsigned long long)stats[i];
    LSM_CUDA(cudaMemcpyAsync(t->d_stats, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    // the host arrays (and the statistics staged above) are read before returning
    LSM_CUDA(cudaStreamSynchronize(st));
    t->n_batches = n_batches;
    return LSM_OK;
}

lsm_status lsm_tally_history_ledger(lsm_tally *t, double *ledger, int64_t n_hist, int64_t first_history)
{
    if (!t) return set_arg_error("lsm_tally_history_ledger: NULL tally");
    if (!ledger) {
        t->hl = nullptr;
        t->hl_n = 0;
        t->hl_g0 = 0;
        return LSM_OK;
    }
    if (t->mode != 0) return set_arg_error("lsm_tally_history_ledger: needs a dose (mode 0) tally");
    if (n_hist < 1 || first_history < 0 || (((uintptr_t)ledger) & 7))
        return set_arg_error("lsm_tally_history_ledger: n_hist >= 1, first_history >= 0, 8-byte aligned buffer");
    t->hl = ledger;
    t->hl_n = n_hist;
    t->hl_g0 = (uint64_t)first_history;
    return LSM_OK;
}

lsm_status lsm_tally_ledger(lsm_tally *t, double ledger[4], int64_t stats[11], lsm_stream stream)
{
    if (!t) return set_arg_error("lsm_tally_ledger: NULL tally");
    RunStats h;
    LSM_CUDA(cudaMemcpyAsync(&h, t->d_stats, sizeof(h), cudaMemcpyDeviceToHost, S(stream)));
    LSM_CUDA(cudaStreamSynchronize(S(stream)));
    if (ledger) for (int i = 0; i < 4; ++i) ledger[i] = h.ledger[i];
    if (stats) for (int i = 0; i < 11; ++i) stats[i] = (int64_t)h.c[i];
    return LSM_OK;
}

lsm_status lsm_transport(const lsm_phantom *ph, const lsm_particles *in, int64_t n, uint64_t seed, lsm_tally *tally,
                         const lsm_run_opts *opts, lsm_stream stream)
{
    return transport_particles(ph, in, n, seed, tally, opts, S(stream));
}

lsm_status lsm_run(const lsm_psl *psl, const lsm_phantom *ph, lsm_tally *tally, uint64_t seed,
                   const lsm_run_opts *opts, lsm_stream stream)
{
    return run_plan(psl, ph, tally, seed, opts, S(stream));
}

lsm_status lsm_dose(const lsm_tally *t, const lsm_phantom *ph, double scale, double *dose, double *sigma, lsm_mem mem,
                    lsm_stream stream)
{
    return dose_impl(t, ph, scale, dose, sigma, mem, S(stream));
}

lsm_status lsm_basis_matrix(const lsm_tally *t, const lsm_psl *psl, const lsm_phantom *ph, const uint16_t *idx3d,
                            lsm_mem idx3d_mem, double *A, lsm_mem mem, lsm_stream stream)
{
    return basis_impl(t, psl, ph, idx3d, idx3d_mem, A, mem, S(stream), false);
}

lsm_status lsm_basis_matrix_units(const lsm_tally *t, const lsm_psl *psl, const lsm_phantom *ph, double *A,
                                  lsm_mem mem, lsm_stream stream)
{
    return basis_impl(t, psl, ph, nullptr, LSM_MEM_DEVICE, A, mem, S(stream), true);
}

lsm_status lsm_model_commission(const lsm_model *model, const double *x, int32_t n_x, lsm_model **out)
{
    return model_commission(model, x, n_x, out);
}

lsm_status lsm_model_weights(const lsm_model *model, double *w) { return model_weights(model, w); }

lsm_status lsm_commission(const double *A, int32_t m, int32_t n, const double *b, lsm_mem mem,
                          const lsm_nnls_opts *opts, double *x, lsm_nnls_report *report, lsm_stream stream)
{
    const int tk = timer_begin(6, S(stream));
    lsm_status rc = commission(A, m, n, b, mem, opts, x, report, S(stream));
    timer_end(tk, S(stream));
    return rc;
}

}  // extern "C"
