// transport.cu -- the sample/transport iteration of Sec. 2.1.3 on the GPU.
//
// Per iteration of M histories:
//   k_sample_queue   steps S3-S5 for M histories; accepted particles that hit
//                    the phantom are compacted by warp ballots into a photon
//                    queue and an electron queue (sub-sources handled apart so
//                    that warps never mix photon and electron code);
//   k_photon         Woodcock tracking of the primary/scatter photons; the two
//                    annihilation photons of a pair event are tracked by the
//                    lane that made them, one after the other;
//   k_electron       CSDA condensed-history electrons;
//   k_flush          FP32 partial tally -> FP64 batch accumulator.
// The transport kernels are persistent: each warp keeps 32 live particles and
// refills a lane from its queue as soon as that lane's particle ends, so warps
// stay full while the queue lasts (the thread-divergence concern of Sec. 2.1.3).
// Particles are regrouped by type (one queue per kind); primary photons are
// also grouped by energy through the sampling loop order (energy bin outer).
// A counting sort of the electron queue by energy cost more than it saved with
// lane refill (electron pass 1.11 -> 0.63 ms per 1e7 histories without it).
//
// The transport physics is the stated simplification of the paper's engine
// (the paper gives only the 200 keV / 50 keV cutoffs, Sec. 2.3): Compton by
// Klein-Nishina (inverse of its closed-form CDF), photoelectric and pair from closed
// forms; electrons by CSDA steps with Bethe stopping power and Highland
// Gaussian deflection. All transport arithmetic is FP32; tallies are flushed
// to FP64.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <string.h>

#include "sample.cuh"

namespace cg = cooperative_groups;

namespace lsm {

struct TP {
    // phantom, local coordinates
    const float *rhomat;
    int nx, ny, nz;
    float inv_dx, inv_dy, inv_dz;
    float lx, ly;              // lateral extent (top face)
    // tables
    const float4 *xs;
    const float *mumax;
    float inv_dlnE, maj;
    // tally: FP32 partials, one slice of `ncell` cells per batch slot
    float *part;
    int64_t ncell;
    const uint16_t *idx;
    int n_rows, n_psr, n_beams;
    // run
    int electron_mode, max_steps;
    float f_e, s_geo;
    const uint32_t *key;       // Philox key (seed) in device memory, so one captured graph serves every seed
    const unsigned *ph_bad;    // nonzero: the phantom's input failed its check (transport does nothing)
    RunStats *stats;
    IterCounters *cnt;
    int ctas_per_sm;           // transport grid: CTAs per SM (0: as many as fit)
    int stage_polls;           // mbarrier polls before a CTA falls back to global-memory tables
    // per-history energy ledger (MODE 2 kernels only): hl[2h] source energy,
    // hl[2h + 1] deposited + escaped + rejected energy of history hl_g0 + h
    double *hl;
    uint64_t hl_g0;
    int64_t hl_n;
};

constexpr int kTableBytes = 2 * kGrid * 16 + kGrid * 4 + kKnE * kKnU * 4;   // 52 KB: photons
constexpr int kXsBytes = 2 * kGrid * 16;                                      // 32 KB: electrons

// resident CTAs per SM the transport kernels are compiled for (register budget)
#ifndef LSM_PHOTON_THREADS
#define LSM_PHOTON_THREADS 256
#endif
// electrons: one CTA of 1024 threads per SM, so that the SM holds one copy of
// the 32 KB tables instead of four and keeps the rest as L1 for the density
// reads (electron pass 0.397 -> 0.391 ms against four CTAs of 256)
#ifndef LSM_ELECTRON_THREADS
#define LSM_ELECTRON_THREADS 1024
#endif
#ifndef LSM_PHOTON_MINB
#define LSM_PHOTON_MINB 3
#endif
#ifndef LSM_ELECTRON_MINB
#define LSM_ELECTRON_MINB 1
#endif
// radiation lengths (g/cm^2): water-like 36.08, bone 21.68

// ---------------------------------------------------------------- tables ---
// CTAs that gave up waiting for their tables (lsm_run_fallbacks)
__device__ unsigned long long g_stage_fallbacks;

// Stage the interaction tables into shared memory with one bulk asynchronous
// copy (cp.async.bulk, completion on an mbarrier). The wait is bounded by
// `polls`; when it runs out the block reports through *err and the fallback
// counter and runs from global memory (drain_stage, before it exits, waits
// for the copy that is still in flight).
template <bool FULL>
__device__ __forceinline__ bool stage_tables(float4 *s_xs, const float4 *g_xs, const float *g_mumax,
                                             uint64_t *mbar, unsigned *err, int polls)
{
    constexpr uint32_t bytes = FULL ? (uint32_t)kTableBytes : (uint32_t)kXsBytes;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(s_xs);
        const uint32_t d1 = (uint32_t)__cvta_generic_to_shared(s_xs + 2 * kGrid);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d0),
            "l"(g_xs), "r"(2 * kGrid * 16), "r"(bar)
            : "memory");
        if (FULL)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d1),
                "l"(g_mumax), "r"(kGrid * 4 + kKnE * kKnU * 4), "r"(bar)
                : "memory");
    }
    __syncthreads();
    uint32_t done = 0;
    for (int it = 0; it < polls && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    }
    const int all = __syncthreads_and(done);
    if (!all && threadIdx.x == 0) {
        atomicOr(err, 1u);
        atomicAdd(&g_stage_fallbacks, 1ull);
    }
    return all != 0;
}

// A CTA that fell back must not exit while its bulk copy may still be writing
// its shared memory: thread 0 waits for the copy to land (at most 2^26 polls;
// the copy of 52 KB takes microseconds).
__device__ __forceinline__ void drain_stage(uint64_t *mbar)
{
    if (threadIdx.x != 0) return;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(mbar);
    uint32_t done = 0;
    for (int it = 0; it < (1 << 26) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    }
}

__device__ __forceinline__ void tab_pos(float inv_dlnE, float E, int &i, float &f)
{
    float t = (__logf(E) - (float)kLnEmin) * inv_dlnE;
    t = fminf(fmaxf(t, 0.0f), (float)(kGrid - 1) - 1e-3f);
    i = (int)t;
    f = t - (float)i;
}

__device__ __forceinline__ float4 lerp4(const float4 *a, int i, float f)
{
    const float4 p = a[i], q = a[i + 1];
    return make_float4(p.x + f * (q.x - p.x), p.y + f * (q.y - p.y), p.z + f * (q.z - p.z),
                       p.w + f * (q.w - p.w));
}

__device__ __forceinline__ int voxel(const TP &T, float x, float y, float z)
{
    const int ix = __float2int_rd(x * T.inv_dx), iy = __float2int_rd(y * T.inv_dy),
              iz = __float2int_rd(z * T.inv_dz);
    if ((unsigned)ix >= (unsigned)T.nx || (unsigned)iy >= (unsigned)T.ny || (unsigned)iz >= (unsigned)T.nz)
        return -1;
    return (iz * T.ny + iy) * T.nx + ix;
}

// A particle's tag word: PSR index (bits 0-15), beam (16-19), batch slot of
// the iteration (20-27). Secondaries inherit it.
__device__ __forceinline__ uint32_t pb_psr(uint32_t pb) { return pb & 0xFFFFu; }
__device__ __forceinline__ uint32_t pb_beam(uint32_t pb) { return (pb >> 16) & 0xFu; }
__device__ __forceinline__ uint32_t pb_slot(uint32_t pb) { return (pb >> 20) & 0xFFu; }
__host__ __device__ __forceinline__ uint32_t pb_make(uint32_t psr, uint32_t beam, uint32_t slot)
{
    return psr | (beam << 16) | (slot << 20);
}

// Compton scattering: v = (eta - 1) / (2k) from the inverse Klein-Nishina CDF
// table, bilinear in (ln E, u); then eta = 1 + 2 k v and cos theta = 1 - 2 v.
__device__ __forceinline__ float kn_inverse(const float *__restrict__ kn, float E, float u)
{
    float t = (__logf(E) - (float)kKnLnE0) * (float)((kKnE - 1) / (kKnLnE1 - kKnLnE0));
    t = fminf(fmaxf(t, 0.0f), (float)(kKnE - 1) - 1e-3f);
    const int i = (int)t;
    const float f = t - (float)i;
    const float sidx = fminf(u * (float)(kKnU - 1), (float)(kKnU - 1) - 1e-4f);
    const int j = (int)sidx;
    const float g = sidx - (float)j;
    const float *a = kn + i * kKnU + j, *b = a + kKnU;
    const float lo = a[0] + g * (a[1] - a[0]), hi = b[0] + g * (b[1] - b[0]);
    return lo + f * (hi - lo);
}

// Compensated FP32 sum (Kahan): the running error of each addition is kept
// in c and subtracted from the next term, so that a thread's sum of a few
// hundred energies stays within a few FP32 roundings of the exact sum. It
// replaces FP64 accumulation in the particle loops, where every FP64
// conversion and add occupies the B300's narrow FP64 pipe for a warp.
struct KSum {
    float s, c;
};
__device__ __forceinline__ void kadd(KSum &k, float x)
{
    const float y = x - k.c;
    const float t = k.s + y;
    k.c = (t - k.s) - y;
    k.s = t;
}
__device__ __forceinline__ double kval(const KSum &k) { return (double)k.s - (double)k.c; }

struct Acc {
    KSum esc, dep;     // escaped energy; deposits of ended particles
    float dep32;       // deposits of the current particle, folded into dep when it ends
    unsigned long long flights, real, esteps, cap;
};

// MODE 0: dose tally; MODE 1: basis tally; MODE 2: dose tally plus the
// per-history energy ledger (a test mode: its own kernel instances, so the
// ledger costs the other modes nothing)
template <int MODE>
__device__ __forceinline__ void hl_add(const TP &T, uint32_t glo, uint32_t ghi, int which, double e)
{
    if constexpr (MODE == 2) {
        const uint64_t h = ((((uint64_t)ghi) << 32) | glo) - T.hl_g0;
        if (h < (uint64_t)T.hl_n) atomicAdd(T.hl + 2 * h + which, e);
    }
}

// FP32 add to a tally cell in L2. KEEP: the line is marked evict-last (an L2
// cache-policy hint), so that the partial slices stay resident while the
// particle queues stream through L2: the photon passes' deposits (local
// electrons below the cutoff, photons below theirs) otherwise miss L2 and their
// line fetches back up the memory pipeline behind the queue traffic (measured
// on the 64^3, 16-slice tally: photon pass 0.65 -> 0.51 ms).
template <bool KEEP>
__device__ __forceinline__ void tally_add(float *cell, float e)
{
    if constexpr (KEEP) {
        uint64_t pol;
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
        asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(cell), "f"(e), "l"(pol) : "memory");
    } else {
        atomicAdd(cell, e);
    }
}

template <int MODE, bool KEEP = false>
__device__ __forceinline__ void deposit(const TP &T, Acc &A, int vox, float e, uint32_t pb, uint32_t glo,
                                        uint32_t ghi)
{
    A.dep32 += e;
    hl_add<MODE>(T, glo, ghi, 1, e);
    float *slice = T.part + (size_t)pb_slot(pb) * T.ncell;
    if (MODE != 1) {
        tally_add<KEEP>(slice + vox, e);
    } else {
        // rows, PSRs and beams are checked so that caller-supplied particles
        // or index arrays can never write outside the basis tally
        const int row = T.idx[vox];
        const uint32_t beam = pb_beam(pb), k = pb_psr(pb);
        if (row && row <= T.n_rows && k < (uint32_t)T.n_psr && beam < (uint32_t)T.n_beams)
            tally_add<KEEP>(slice + ((size_t)beam * T.n_rows + (row - 1)) * T.n_psr + k, e);
    }
}

// rotate (u, v, w) by polar cos(theta) and azimuth 2 pi uphi
__device__ __forceinline__ void rotate(float &u, float &v, float &w, float cost, float uphi)
{
    const float sint = sqrtf(fmaxf(0.0f, 1.0f - cost * cost));
    float sp, cp;
    __sincosf(6.28318531f * uphi, &sp, &cp);
    float un, vn, wn;
    if (fabsf(w) < 0.99999f) {
        const float q = 1.0f - w * w, is = rsqrtf(q), s = q * is;
        un = u * cost + sint * (u * w * cp - v * sp) * is;
        vn = v * cost + sint * (v * w * cp + u * sp) * is;
        wn = w * cost - sint * s * cp;
    } else {
        un = sint * cp;
        vn = sint * sp;
        wn = (w > 0.0f ? 1.0f : -1.0f) * cost;
    }
    const float in = rsqrtf(un * un + vn * vn + wn * wn);
    u = un * in; v = vn * in; w = wn * in;
}

// An electron a photon created during its step, pushed by the whole warp
// after the step (one queue reservation serves many pushes).
struct Pend {
    float x, y, z, u, v, w, E;
    uint32_t sid;
    int vox;
};

// The second annihilation photon of a pair event,
// transported by the same lane after the first one (both start at the pair
// vertex; position, direction and stream id).
struct Ann {
    float x, y, z, u, v, w;
    uint32_t sid;
};

struct Part {
    float x, y, z, u, v, w, E;
    Stream rng;
    uint32_t pb;
    int steps;
    int vc;        // electrons: voxel whose (sign-coded) density is held in rc, -1 if none
    float rc;
    int dv;        // electrons: voxel of the deposit not yet written, -1 if none
    float de;      // and its energy (consecutive steps in one voxel add up here)
};

__device__ __forceinline__ void load_part(const Queue &q, uint32_t i, uint32_t k0, uint32_t k1, Part &p)
{
    const float4 a = q.rec[3 * (size_t)i], b = q.rec[3 * (size_t)i + 1], c = q.rec[3 * (size_t)i + 2];
    p.x = a.x; p.y = a.y; p.z = a.z; p.E = a.w;
    p.u = b.x; p.v = b.y; p.w = b.z;
    p.rng.k0 = k0; p.rng.k1 = k1;
    p.rng.glo = __float_as_uint(c.x); p.rng.ghi = __float_as_uint(c.y); p.rng.sid = __float_as_uint(b.w);
    p.rng.ctr = 0;
    p.pb = __float_as_uint(c.z);
    p.steps = 0;
    p.vc = -1;
    p.rc = 0.0f;
    p.dv = -1;
    p.de = 0.0f;
    p.rng.have = 0;
}

__device__ __forceinline__ void store_part(const Queue &q, uint32_t i, float x, float y, float z, float u,
                                           float v, float w, float E, uint32_t glo, uint32_t ghi, uint32_t sid,
                                           uint32_t pb)
{
    float4 *r = q.rec + 3 * (size_t)i;
    r[0] = make_float4(x, y, z, E);
    r[1] = make_float4(u, v, w, __uint_as_float(sid));
    r[2] = make_float4(__uint_as_float(glo), __uint_as_float(ghi), __uint_as_float(pb), 0.0f);
}

// Append one particle from divergent code: one atomic per coalesced group.
__device__ __forceinline__ uint32_t push_slot(uint32_t *counter)
{
    cg::coalesced_group g = cg::coalesced_threads();
    uint32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (uint32_t)g.size());
    base = g.shfl(base, 0);
    return base + g.thread_rank();
}

// An electron entering the phantom from the source (or a caller's particle
// list): queued, or, when the electron queue is full (a run with a small
// e_queue_cap), deposited in the voxel where it enters and counted.
template <int MODE>
__device__ __forceinline__ void enqueue_source_electron(const TP &T, Acc &A, const Queue &eq, uint32_t slot, float lx,
                                                        float ly, float lz, float u, float v, float w, float E,
                                                        uint32_t glo, uint32_t ghi, uint32_t pb)
{
    if (slot < eq.cap) {
        store_part(eq, slot, lx, ly, lz, u, v, w, E, glo, ghi, 1u, pb);
    } else {
        atomicAdd(&T.stats->c[9], 1ull);
        deposit<MODE>(T, A, voxel(T, lx, ly, lz), E, pb, glo, ghi);
    }
}

template <int MODE>
__device__ __forceinline__ void spawn_electron(const TP &T, Acc &A, const Queue &eq, const Part &p, float Te,
                                               float u, float v, float w, uint32_t sid, int vox)
{
    if (T.electron_mode == 0 || Te < kCutE) {
        deposit<MODE, true>(T, A, vox, Te, p.pb, p.rng.glo, p.rng.ghi);
        return;
    }
    const uint32_t slot = push_slot(&T.cnt->n[2]);
    if (slot >= eq.cap) {
        atomicAdd(&T.stats->c[9], 1ull);
        deposit<MODE, true>(T, A, vox, Te, p.pb, p.rng.glo, p.rng.ghi);
        return;
    }
    store_part(eq, slot, p.x, p.y, p.z, u, v, w, Te, p.rng.glo, p.rng.ghi, sid, p.pb);
}

// One Woodcock flight (and the interaction if the collision is real), on one
// Philox block: word 0 -> flight length, word 1 -> the collision (virtual, or
// which interaction), words 2-3 -> a Compton event's eta and azimuth; a pair
// event draws one more block. Returns false when the photon's history ends.
template <int MODE>
__device__ bool photon_step(const TP &T, const float4 *xs, const float *mumax_t, Acc &A, Part &p,
                            const Queue &eq, Pend &pe, bool &pend, Ann &an, bool &ann)
{
    // A photon starts a flight inside the phantom with E at or above the
    // cutoff: queued photons are checked where a lane loads them, a flight
    // that leaves the phantom ends the photon, and a Compton event that takes
    // E below the cutoff deposits it at once. So the top of a flight needs no
    // voxel lookup (one per flight fewer: photon pass 0.441 -> 0.426 ms).
    if (++p.steps > T.max_steps) {
        A.cap++;
        deposit<MODE, true>(T, A, voxel(T, p.x, p.y, p.z), p.E, p.pb, p.rng.glo, p.rng.ghi);
        return false;
    }
    const uint4 r = p.rng.next();
    int ti;
    float tf;
    tab_pos(T.inv_dlnE, p.E, ti, tf);
    const float mm = (mumax_t[ti] + tf * (mumax_t[ti + 1] - mumax_t[ti])) * T.maj;
    const float s = __fdividef(-__logf(u01(r.x)), mm);
    p.x += s * p.u; p.y += s * p.v; p.z += s * p.w;
    A.flights++;
    const int vox = voxel(T, p.x, p.y, p.z);
    if (vox < 0) { kadd(A.esc, p.E); hl_add<MODE>(T, p.rng.glo, p.rng.ghi, 1, p.E); return false; }
    const float rm = __ldg(T.rhomat + vox);
    // the block of the next draw (next flight, or a pair event's) does not
    // depend on the density: compute it while the load is in flight
    p.rng.prefetch();
    const int m = rm < 0.0f;
    const float rho = fabsf(rm);
    const float4 c = lerp4(xs + m * kGrid, ti, tf);
    const float muC = c.x * rho, muP = c.y * rho, muQ = c.z * rho;
    const float mut = muC + muP + muQ;
    // t is uniform on [0, mm): above mut the collision is virtual, below it t
    // is uniform on [0, mut) and picks the interaction
    const float t = u01(r.y) * mm;
    if (t > mut) return true;                                   // virtual collision
    A.real++;
    if (t <= muC) {
        // Compton: word 2 -> E'/E by the inverse Klein-Nishina CDF, word 3 -> azimuth
        const float k = p.E * (1.0f / kMe);
        const float vkn = kn_inverse(mumax_t + kGrid, p.E, u01(r.z));
        const float eta = 1.0f + 2.0f * k * vkn;
        const float cost = 1.0f - 2.0f * vkn;
        const float E1 = __fdividef(p.E, eta);
        const float uphi = u01(r.w);
        float u = p.u, v = p.v, w = p.w;
        rotate(u, v, w, cost, uphi);
        float ex = p.E * p.u - E1 * u, ey = p.E * p.v - E1 * v, ez = p.E * p.w - E1 * w;
        const float en2 = ex * ex + ey * ey + ez * ez;
        if (en2 > 0.0f) { const float in = rsqrtf(en2); ex *= in; ey *= in; ez *= in; }
        else { ex = p.u; ey = p.v; ez = p.w; }
        const float Te = p.E - E1;
        if (T.electron_mode && Te >= kCutE) {
            pe = Pend{p.x, p.y, p.z, ex, ey, ez, Te, p.rng.child_id(0), vox};
            pend = true;
        } else {
            deposit<MODE, true>(T, A, vox, Te, p.pb, p.rng.glo, p.rng.ghi);
        }
        if (E1 < kCutG) { deposit<MODE, true>(T, A, vox, E1, p.pb, p.rng.glo, p.rng.ghi); return false; }
        p.E = E1; p.u = u; p.v = v; p.w = w;
        return true;
    }
    if (t <= muC + muP) {
        // photoelectric: the electron takes the photon's energy and direction
        if (T.electron_mode && p.E >= kCutE) {
            pe = Pend{p.x, p.y, p.z, p.u, p.v, p.w, p.E, p.rng.child_id(0), vox};
            pend = true;
        } else {
            deposit<MODE, true>(T, A, vox, p.E, p.pb, p.rng.glo, p.rng.ghi);
        }
        return false;
    }
    // pair: uniform kinetic split, leptons along the photon; annihilation
    // photons leave the interaction point back to back, isotropic
    const uint4 q = p.rng.next();
    const float Tk = p.E - 2.0f * kMe;
    const float Tm = u01(q.x) * Tk, Tp = Tk - Tm;
    const float ca = 2.0f * u01(q.y) - 1.0f;
    const float sa = sqrtf(fmaxf(0.0f, 1.0f - ca * ca));
    float sp, cp;
    sincospif(2.0f * u01(q.z), &sp, &cp);
    const float ax = sa * cp, ay = sa * sp, az = ca;
    spawn_electron<MODE>(T, A, eq, p, Tm, p.u, p.v, p.w, p.rng.child_id(0), vox);
    spawn_electron<MODE>(T, A, eq, p, Tp, p.u, p.v, p.w, p.rng.child_id(1), vox);
    // the lane goes on with the first annihilation photon and keeps the second
    // for after it (a queue of their own and a pass over it was latency-bound
    // on a few ten thousand photons: 0.032 ms of a 1.24 ms step)
    an = Ann{p.x, p.y, p.z, -ax, -ay, -az, p.rng.child_id(3)};
    ann = true;
    p.rng.sid = p.rng.child_id(2);
    p.rng.ctr = 0;
    p.rng.have = 0;
    p.E = kMe;
    p.u = ax; p.v = ay; p.w = az;
    p.steps = 0;
    return true;
}

// An electron deposits about twice per voxel: deposits into the voxel of the
// previous one are added in a register and written when the voxel changes or
// the electron ends.
template <int MODE>
__device__ __forceinline__ void edep(const TP &T, Acc &A, Part &p, int vox, float e)
{
    if (vox == p.dv) { p.de += e; return; }
    if (p.dv >= 0) deposit<MODE>(T, A, p.dv, p.de, p.pb, p.rng.glo, p.rng.ghi);
    p.dv = vox;
    p.de = e;
}

template <int MODE>
__device__ __forceinline__ void eflush(const TP &T, Acc &A, Part &p)
{
    if (p.dv >= 0) deposit<MODE>(T, A, p.dv, p.de, p.pb, p.rng.glo, p.rng.ghi);
    p.dv = -1;
}

// One CSDA step. Returns false when the electron's history ends.
template <int MODE>
__device__ bool electron_step(const TP &T, const float4 *xs, Acc &A, Part &p, const uint4 &blk, bool &blk_used)
{
    // (reusing the previous step's end voxel here measured 1.6x slower)
    const int vox = voxel(T, p.x, p.y, p.z);
    if (vox < 0) { eflush<MODE>(T, A, p); kadd(A.esc, p.E); hl_add<MODE>(T, p.rng.glo, p.rng.ghi, 1, p.E); return false; }
    if (p.E < kCutE) { edep<MODE>(T, A, p, vox, p.E); eflush<MODE>(T, A, p); return false; }
    if (++p.steps > T.max_steps) {
        A.cap++;
        edep<MODE>(T, A, p, vox, p.E);
        eflush<MODE>(T, A, p);
        return false;
    }
    // an electron takes about two steps per voxel: reuse the density loaded
    // for this voxel at the end of the previous step
    const float rm = vox == p.vc ? p.rc : __ldg(T.rhomat + vox);
    const int m = rm < 0.0f;
    const float rho = fabsf(rm);
    int ti;
    float tf;
    tab_pos(T.inv_dlnE, p.E, ti, tf);
    const float4 c0 = lerp4(xs + m * kGrid, ti, tf);
    const float S = c0.w * rho;
    const float ds = fminf(__fdividef(T.f_e * p.E, S), T.s_geo);
    const float Emid = p.E - 0.5f * S * ds;               // midpoint rule
    tab_pos(T.inv_dlnE, Emid, ti, tf);
    const float4 c1 = lerp4(xs + m * kGrid, ti, tf);
    const float dE = fminf(c1.w * rho * ds, p.E);
    const float hs = 0.5f * ds;
    const int vm = voxel(T, p.x + hs * p.u, p.y + hs * p.v, p.z + hs * p.w);
    if (vm >= 0) edep<MODE>(T, A, p, vm, dE);
    else { kadd(A.esc, dE); hl_add<MODE>(T, p.rng.glo, p.rng.ghi, 1, dE); }
    A.esteps++;
    const float E0 = p.E;
    p.x += ds * p.u; p.y += ds * p.v; p.z += ds * p.w;
    p.E -= dE;
    // issue the next voxel's density load now, so that it is in flight while
    // the deflection below is computed
    const int vn = voxel(T, p.x, p.y, p.z);
    p.rc = vn == vox ? rm : (vn >= 0 ? __ldg(T.rhomat + vn) : 0.0f);
    p.vc = vn;
    if (p.E >= kCutE) {
        // one block serves two deflections: words 0-1, then words 2-3 (held in
        // pre while `have` is set; electrons never prefetch blocks)
        float ua, ub;
        if (p.rng.have) {
            ua = u01(p.rng.pre.z);
            ub = u01(p.rng.pre.w);
            p.rng.have = 0;
        } else {
            // the block at the stream's counter, computed by the caller for
            // the warp's two steps at once (one of them needs it at most)
            uint4 r;
            if (!blk_used) {
                r = blk;
                ++p.rng.ctr;
                blk_used = true;
            } else {
                r = p.rng.next();
            }
            ua = u01(r.x);
            ub = u01(r.y);
            p.rng.pre = r;
            p.rng.have = 1;
        }
        const float t = rho * ds * (m ? (1.0f / 21.68f) : (1.0f / 36.08f));
        // Highland width: 13.6 MeV / (beta c p) sqrt(t) (1 + 0.038 ln t), beta c p = E(E + 2m)/(E + m)
        const float f = fmaxf(1.0f + 0.038f * __logf(t), 0.0f);
        const float th0 = __fdividef(13.6f * (E0 + kMe), E0 * (E0 + 2.0f * kMe)) * sqrtf(t) * f;
        const float th = fminf(th0 * sqrtf(-2.0f * __logf(ua)), kPi);
        rotate(p.u, p.v, p.w, __cosf(th), ub);
    }
    return true;
}

__device__ void flush_acc(const TP &T, const Acc &A)
{
    const double esc = warp_sum(kval(A.esc)), dep = warp_sum(kval(A.dep) + (double)A.dep32);
    const unsigned long long fl = warp_sum_u64(A.flights), re = warp_sum_u64(A.real),
                             es = warp_sum_u64(A.esteps), cp = warp_sum_u64(A.cap);
    if (lane_id() == 0) {
        if (esc != 0.0) atomicAdd(&T.stats->ledger[2], esc);
        if (dep != 0.0) atomicAdd(&T.stats->ledger[3], dep);
        if (fl) atomicAdd(&T.stats->c[5], fl);
        if (re) atomicAdd(&T.stats->c[6], re);
        if (es) atomicAdd(&T.stats->c[7], es);
        if (cp) atomicAdd(&T.stats->c[8], cp);
    }
}

// Persistent transport kernel with per-lane refill from queue `qi`.
// KIND 0: photons (Woodcock), KIND 1: electrons (CSDA).
template <int MODE, int KIND>
__global__ void __launch_bounds__(KIND ? LSM_ELECTRON_THREADS : LSM_PHOTON_THREADS,
                                  KIND ? LSM_ELECTRON_MINB : LSM_PHOTON_MINB) k_transport(TP T, Queue in, int qi, Queue eq)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    const uint32_t n_q = *(volatile uint32_t *)&T.cnt->n[qi];
    const uint32_t n_in = n_q < in.cap ? n_q : in.cap;     // pushes beyond capacity were not stored
    const uint32_t k0 = T.key[0], k1 = T.key[1];
    if (KIND == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
        // the photon pass is complete: the electron queue holds the source's
        // electrons, the secondaries of photon interactions and dead slots
        const uint32_t other = T.cnt->src_e + T.cnt->dead;
        if (n_in > other) atomicAdd(&T.stats->c[10], (unsigned long long)(n_in - other));
    }
    // blocks whose first slot lies past the queue end have nothing to refill
    // from once the earlier blocks start: leave before staging the tables; a
    // phantom whose input failed its check (a creation that left the check to
    // the device) is not transported through
    if ((uint64_t)blockIdx.x * blockDim.x >= n_in || *(volatile const unsigned *)T.ph_bad) return;
    float4 *s_xs = reinterpret_cast<float4 *>(smem);
    float *s_mm = reinterpret_cast<float *>(smem + 2 * kGrid * 16);
    const bool staged = stage_tables<KIND == 0>(s_xs, T.xs, T.mumax, &mbar, &T.cnt->pad, T.stage_polls);
    const float4 *xs = staged ? s_xs : T.xs;
    const float *mm = staged ? s_mm : T.mumax;
    uint32_t *head = &T.cnt->head[qi];
    const unsigned lane = lane_id();
    unsigned lt;
    lanemask_lt(lt);
    Acc A = {{0.0f, 0.0f}, {0.0f, 0.0f}, 0.0f, 0ull, 0ull, 0ull, 0ull};
    Part p;
    bool alive = false;
    // Each warp reserves kGrab consecutive queue slots per atomic and hands
    // them to its lanes as they fall idle; [rb, rb + rl) is the unused part
    // of the reservation (warp-uniform). Slots are handed out in queue order,
    // so once a handed-out slot lies past the end, every later one does too.
#ifndef LSM_GRAB_DIV
#define LSM_GRAB_DIV 8
#endif
    // a reservation is 32-256 slots, about 1/LSM_GRAB_DIV of a warp's share of
    // the queue: few enough atomics and long enough prefetch lead, fine enough
    // that the queue's end leaves little imbalance
    const uint32_t share = n_in / (gridDim.x * (blockDim.x >> 5) * LSM_GRAB_DIV);
    const uint32_t kGrab = share >= 256 ? 256u : (share >= 128 ? 128u : (share >= 64 ? 64u : 32u));
    uint32_t rb = 0, rl = 0;
    bool exhausted = false;
    Ann an = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0u};
    bool ann = false;
    // output reservation for the electrons photons create: [ob, ob + ol);
    // 64 slots per atomic (32: photon pass 0.47 -> 0.49 ms; 128: the dead
    // entries left at the end slow the electron pass by more than it gains)
    constexpr uint32_t kOut = 64;
    uint32_t ob = 0, ol = 0;
    for (;;) {
        const unsigned need = __ballot_sync(0xffffffffu, !alive);
        const uint32_t k = (uint32_t)__popc(need);
        if (k && (rl > 0 || !exhausted)) {
            uint32_t nb = 0;
            bool grabbed = false;
            if (rl < k && !exhausted) {
                if (lane == 0) {
                    // read before the atomic: once the queue is exhausted, warps stop hammering its cursor
                    const uint32_t h = *(volatile uint32_t *)head;
                    nb = h >= n_in ? n_in : atomicAdd(head, kGrab);
                }
                nb = __shfl_sync(0xffffffffu, nb, 0);
                grabbed = true;
                if (nb + kGrab >= n_in) exhausted = true;
                // the reservation's records are handed out over the next few
                // steps: start moving them from DRAM into L2 now (one 128-byte
                // line per lane, inside the queue's filled part)
                if (nb < n_in) {
                    const size_t bytes = (size_t)(min(nb + kGrab, n_in) - nb) * 48;
                    const size_t off = (size_t)lane * 128;
                    if (off < bytes)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"((const char *)(in.rec + 3 * (size_t)nb) + off));
                }
            }
            if (!alive) {
                const uint32_t r = (uint32_t)__popc(need & lt);
                const uint32_t i = r < rl ? rb + r : (grabbed ? nb + (r - rl) : 0xffffffffu);
                if (i < n_in) {
                    load_part(in, i, k0, k1, p);
                    alive = true;
                    // queued photons lie inside the phantom; one below the
                    // photon cutoff (a caller's particle) deposits where it is
                    if (KIND == 0 && p.E < kCutG) {
                        deposit<MODE, true>(T, A, voxel(T, p.x, p.y, p.z), p.E, p.pb, p.rng.glo, p.rng.ghi);
                        kadd(A.dep, A.dep32);
                        A.dep32 = 0.0f;
                        alive = false;
                    }
                }
            }
            if (grabbed) {
                const uint32_t from_new = k - rl;
                rb = nb + from_new;
                rl = kGrab - from_new;
            } else {
                rb += k;
                rl = rl > k ? rl - k : 0;
            }
        }
        if (KIND == 0 && rl > 0 && rb < n_in) {
            // the records the next refills take (the next 32 slots of the
            // reservation, already in L2): one L1 prefetch per 128-byte line,
            // so that a refilled lane's first flight does not wait on L2
            // (photon pass 0.426 -> 0.421 ms; on the electron pass it cost
            // 0.39 -> 0.405 ms, so electrons do without)
            const uint32_t nrec = min(min(rl, 32u), n_in - rb);
            const size_t line = (((size_t)rb * 48) >> 7) + lane;
            if (line <= ((((size_t)rb + nrec) * 48 - 1) >> 7))
                asm volatile("prefetch.global.L1 [%0];" ::"l"((const char *)in.rec + (line << 7)));
        }
        if (!__any_sync(0xffffffffu, alive)) break;
        if constexpr (KIND == 1) {
            if (alive) {
                // two CSDA steps per pass of the loop: each consumes two words
                // of a Philox block, so together they need at most one new
                // block, computed here for all live lanes at once instead of
                // by whichever lanes happen to need one at each step
                const uint4 blk = philox4x32_10(p.rng.k0, p.rng.k1, p.rng.glo, p.rng.ghi, p.rng.sid, p.rng.ctr);
                bool used = false;
                alive = electron_step<MODE>(T, xs, A, p, blk, used);
                if (alive) alive = electron_step<MODE>(T, xs, A, p, blk, used);
                if (!alive) { kadd(A.dep, A.dep32); A.dep32 = 0.0f; }
            }
        } else {
            bool pend = false;
            Pend pe;
            const uint32_t pb_keep = p.pb;
            if (alive) {
                alive = photon_step<MODE>(T, xs, mm, A, p, eq, pe, pend, an, ann);
                if (!alive) {
                    kadd(A.dep, A.dep32);
                    A.dep32 = 0.0f;
                    if (ann) {
                        // the pair's second annihilation photon, same history and tag
                        p.x = an.x; p.y = an.y; p.z = an.z;
                        p.u = an.u; p.v = an.v; p.w = an.w;
                        p.E = kMe;
                        p.rng.sid = an.sid;
                        p.rng.ctr = 0;
                        p.rng.have = 0;
                        p.steps = 0;
                        ann = false;
                        alive = true;
                    }
                }
            }
            // warp-wide push of the electrons created in this step
            const unsigned pm = __ballot_sync(0xffffffffu, pend);
            if (pm) {
                const uint32_t n = (uint32_t)__popc(pm);
                uint32_t nb = 0;
                bool g2 = false;
                if (ol < n) {
                    if (lane == 0) nb = atomicAdd(&T.cnt->n[2], kOut);
                    nb = __shfl_sync(0xffffffffu, nb, 0);
                    g2 = true;
                }
                if (pend) {
                    const uint32_t r = (uint32_t)__popc(pm & lt);
                    const uint32_t slot = r < ol ? ob + r : nb + (r - ol);
                    if (slot < eq.cap) {
                        store_part(eq, slot, pe.x, pe.y, pe.z, pe.u, pe.v, pe.w, pe.E, p.rng.glo, p.rng.ghi, pe.sid,
                                   pb_keep);
                    } else {
                        atomicAdd(&T.stats->c[9], 1ull);
                        deposit<MODE, true>(T, A, pe.vox, pe.E, pb_keep, p.rng.glo, p.rng.ghi);
                        kadd(A.dep, A.dep32);
                        A.dep32 = 0.0f;
                    }
                }
                if (g2) {
                    const uint32_t from_new = n - ol;
                    ob = nb + from_new;
                    ol = kOut - from_new;
                } else {
                    ob += n;
                    ol -= n;
                }
            }
        }
    }
    if (KIND == 0 && ol) {
        // reserved output slots this warp did not fill hold dead entries
        // (outside the phantom, no energy) that the electron kernel discards
        for (uint32_t j = lane; j < ol; j += 32)
            if (ob + j < eq.cap)
                store_part(eq, ob + j, -1.0f, -1.0f, -1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0u, 0u, 2u, 0u);
        if (lane == 0 && ob < eq.cap) atomicAdd(&T.cnt->dead, min(ol, eq.cap - ob));
    }
    flush_acc(T, A);
    if (!staged) drain_stage(&mbar);
}

// ------------------------------------------------------------ sampling ---

struct SQ {
    SampleParams sp;
    const uint32_t *key;    // Philox key in device memory
    uint64_t g0;            // history of the iteration's first particle
    int64_t h0, n;          // its plan position; histories in the iteration
    int64_t plan;           // plan size: position h0 + i lies in batch slot (h0 + i) / plan
    float z_rel;            // phantom surface - z_phsp
    float x0, y0;           // phantom corner on the surface plane
    float z0, lz;           // phantom corner z and depth (rotated beams)
};

// Rotated beams: the particle's ray from the phase-space plane, turned into
// phantom coordinates about the isocentre, meets the voxel box [0, lx] x
// [0, ly] x [0, lz] (slab method); the particle starts 1e-4 cm past the entry
// point. Returns false when the ray misses the box. Phantom-local position
// and direction out.
__device__ __forceinline__ bool enter_box(const SQ &S, const TP &T, const SrcParticle &o, float &px, float &py,
                                          float &pz, float &du, float &dv, float &dw)
{
    const float2 cs = __ldg(S.sp.rot + o.beam);
    const float qz = S.sp.z_phsp - S.sp.sad;                 // plane relative to the isocentre
    const float p0 = S.sp.iso[0] + o.xp * cs.x + qz * cs.y - S.x0;
    const float p1 = S.sp.iso[1] + o.yp - S.y0;
    const float p2 = S.sp.iso[2] - o.xp * cs.y + qz * cs.x - S.z0;
    du = o.u * cs.x + o.w * cs.y;
    dv = o.v;
    dw = o.w * cs.x - o.u * cs.y;
    const float p[3] = {p0, p1, p2}, d[3] = {du, dv, dw}, L[3] = {T.lx, T.ly, S.lz};
    float tn = 0.0f, tf = 3.0e38f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            const float id = 1.0f / d[a];
            const float t1 = (0.0f - p[a]) * id, t2 = (L[a] - p[a]) * id;
            tn = fmaxf(tn, fminf(t1, t2));
            tf = fminf(tf, fmaxf(t1, t2));
        } else if (p[a] < 0.0f || p[a] > L[a]) {
            tf = -1.0f;
        }
    }
    if (!(tn <= tf)) return false;
    const float t = tn + 1e-4f;
    px = p0 + t * du;
    py = p1 + t * dv;
    pz = p2 + t * dw;
    return voxel(T, px, py, pz) >= 0;
}

template <int MODE>
__global__ void __launch_bounds__(256) k_sample_queue(SQ S, TP T, Queue pq, Queue eq)
{
    // a plan whose sampling areas hold no weight has no entries: nothing to
    // sample (the host reports it when it reads the plan's results)
    const int64_t n_ent = __ldg(S.sp.n_ent);
    if (n_ent < 1) return;
    const uint32_t k0 = S.key[0], k1 = S.key[1];
    const unsigned lane = lane_id();
    unsigned lt;
    lanemask_lt(lt);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // source, rejected and missed energy per thread in FP64: the source
    // energy is the same sum, to FP64 rounding, however the run is split
    double src = 0.0, rej = 0.0, esc = 0.0;
    Acc A = {{0.0f, 0.0f}, {0.0f, 0.0f}, 0.0f, 0ull, 0ull, 0ull, 0ull};
    unsigned long long nph = 0, nel = 0, nrej = 0, nmiss = 0;
    // batch slot and plan position of this lane's history, (h0 + i) / plan and
    // its remainder, advanced by the loop's stride without a 64-bit division
    // per history
    const int64_t stride = nwarps * 32;
    const int64_t q_st = stride / S.plan, r_st = stride - q_st * S.plan;
    int64_t slot_l = (S.h0 + warp * 32 + lane) / S.plan;
    int64_t hpos_l = S.h0 + warp * 32 + lane - slot_l * S.plan;
    for (int64_t base = warp * 32; base < S.n; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < S.n;
        SrcParticle o;
        o.stype = 0;
        bool in = false;
        float lx = 0.0f, ly = 0.0f, lz = 0.0f;
        const uint32_t slot = valid ? (uint32_t)slot_l : 0u;
        const int64_t hpos = hpos_l;
        hpos_l += r_st;
        slot_l += q_st;
        if (hpos_l >= S.plan) { hpos_l -= S.plan; ++slot_l; }
        const int64_t ek = find_entry_warp(S.sp.start, n_ent, hpos, valid);
        if (valid) {
            sample_history(S.sp, k0, k1, S.g0 + (uint64_t)i, hpos, S.z_rel, o, ek);
            const uint64_t gh = S.g0 + (uint64_t)i;
            src += o.E;
            hl_add<MODE>(T, (uint32_t)gh, (uint32_t)(gh >> 32), 0, o.E);
            if (!o.accepted) { rej += o.E; nrej++; hl_add<MODE>(T, (uint32_t)gh, (uint32_t)(gh >> 32), 1, o.E); }
            else {
                if (!S.sp.rotated) {
                    lx = o.x - S.x0; ly = o.y - S.y0;
                    in = voxel(T, lx, ly, 0.0f) >= 0;   // crosses the phantom's top face
                } else {
                    float du, dv, dw;
                    in = enter_box(S, T, o, lx, ly, lz, du, dv, dw);
                    o.u = du; o.v = dv; o.w = dw;
                }
                if (!in) { esc += o.E; nmiss++; hl_add<MODE>(T, (uint32_t)gh, (uint32_t)(gh >> 32), 1, o.E); }
            }
        }
        const bool is_e = o.stype == 2;
        const bool local_e = in && is_e && T.electron_mode == 0;
        const unsigned mp = __ballot_sync(0xffffffffu, in && !is_e);
        const unsigned me = __ballot_sync(0xffffffffu, in && is_e && !local_e);
        uint32_t bp = 0, be = 0;
        if (lane == 0) {
            if (mp) bp = atomicAdd(&T.cnt->n[0], (uint32_t)__popc(mp));
            if (me) {
                be = atomicAdd(&T.cnt->n[2], (uint32_t)__popc(me));
                atomicAdd(&T.cnt->src_e, (uint32_t)__popc(me));
            }
        }
        bp = __shfl_sync(0xffffffffu, bp, 0);
        be = __shfl_sync(0xffffffffu, be, 0);
        if (in) {
            const uint64_t g = S.g0 + (uint64_t)i;
            const uint32_t pb = pb_make((uint32_t)o.psr, (uint32_t)o.beam, slot);
            if (!is_e) {
                nph++;
                store_part(pq, bp + __popc(mp & lt), lx, ly, lz, o.u, o.v, o.w, o.E, (uint32_t)g,
                           (uint32_t)(g >> 32), 1u, pb);
            } else {
                nel++;
                if (local_e) {
                    deposit<MODE>(T, A, voxel(T, lx, ly, lz), o.E, pb, (uint32_t)g, (uint32_t)(g >> 32));
                } else {
                    enqueue_source_electron<MODE>(T, A, eq, be + __popc(me & lt), lx, ly, lz, o.u, o.v, o.w, o.E,
                                                  (uint32_t)g, (uint32_t)(g >> 32), pb);
                }
            }
        }
    }
    const double src_d = warp_sum(src), rej_d = warp_sum(rej), esc_d = warp_sum(esc);
    const double dep = warp_sum(kval(A.dep) + (double)A.dep32);
    nph = warp_sum_u64(nph); nel = warp_sum_u64(nel); nrej = warp_sum_u64(nrej); nmiss = warp_sum_u64(nmiss);
    if (lane == 0) {
        atomicAdd(&T.stats->ledger[0], src_d);
        if (rej_d != 0.0) atomicAdd(&T.stats->ledger[1], rej_d);
        if (esc_d != 0.0) atomicAdd(&T.stats->ledger[2], esc_d);
        if (dep != 0.0) atomicAdd(&T.stats->ledger[3], dep);
        if (nph) atomicAdd(&T.stats->c[1], nph);
        if (nel) atomicAdd(&T.stats->c[2], nel);
        if (nrej) atomicAdd(&T.stats->c[3], nrej);
        if (nmiss) atomicAdd(&T.stats->c[4], nmiss);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&T.stats->c[0], (unsigned long long)S.n);
}

// Public sampler: one record per history (global coordinates).
__global__ void k_sample_public(SampleParams sp, uint32_t k0, uint32_t k1, uint64_t g0, int64_t h0,
                                int64_t plan_size, int64_t n, float z_rel, float z_surf, lsm_particles out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int64_t h = h0 + i;
        if (h >= plan_size) h %= plan_size;
        SrcParticle o;
        sample_history(sp, k0, k1, g0 + (uint64_t)i, h, z_rel, o);
        out.x[i] = o.x; out.y[i] = o.y; out.z[i] = z_surf;
        out.u[i] = o.u; out.v[i] = o.v; out.w[i] = o.w; out.E[i] = o.E;
        out.hist[i] = g0 + (uint64_t)i;
        out.psr[i] = (uint16_t)o.psr;
        out.beam[i] = (uint8_t)o.beam;
        out.type[i] = o.stype == 2 ? 1 : 0;
        out.status[i] = o.accepted ? 0 : 1;
        if (out.info) {
            int32_t *q = out.info + 4 * i;
            q[0] = o.stype | (o.ebin << 8);
            q[1] = o.ring;
            q[2] = o.comp;
            q[3] = (int32_t)o.entry;
        }
    }
}

// Load caller-provided particles (global coordinates) into the queues.
template <int MODE>
__global__ void k_enqueue(lsm_particles P, int64_t n, float x0, float y0, float z0, TP T, Queue pq, Queue eq)
{
    const unsigned lane = lane_id();
    unsigned lt;
    lanemask_lt(lt);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double esc = 0.0;
    Acc A = {{0.0f, 0.0f}, {0.0f, 0.0f}, 0.0f, 0ull, 0ull, 0ull, 0ull};
    unsigned long long nph = 0, nel = 0, nmiss = 0;
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const int64_t i = base + lane;
        bool is_e = false, inside = false;
        float lx = 0, ly = 0, lz = 0;
        if (i < n && P.status[i] == 0) {
            is_e = P.type[i] == 1;
            lx = P.x[i] - x0; ly = P.y[i] - y0; lz = P.z[i] - z0;
            inside = lx >= 0.0f && lx < T.lx && ly >= 0.0f && ly < T.ly && lz >= 0.0f &&
                     voxel(T, lx, ly, lz) >= 0;
            if (!inside) { esc += P.E[i]; nmiss++; }
        }
        const bool local_e = inside && is_e && T.electron_mode == 0;
        const unsigned mp = __ballot_sync(0xffffffffu, inside && !is_e);
        const unsigned me = __ballot_sync(0xffffffffu, inside && is_e && !local_e);
        uint32_t bp = 0, be = 0;
        if (lane == 0) {
            if (mp) bp = atomicAdd(&T.cnt->n[0], (uint32_t)__popc(mp));
            if (me) {
                be = atomicAdd(&T.cnt->n[2], (uint32_t)__popc(me));
                atomicAdd(&T.cnt->src_e, (uint32_t)__popc(me));
            }
        }
        bp = __shfl_sync(0xffffffffu, bp, 0);
        be = __shfl_sync(0xffffffffu, be, 0);
        if (inside) {
            const uint64_t g = P.hist[i];
            const uint32_t pb = pb_make((uint32_t)P.psr[i], (uint32_t)P.beam[i] & 0xFu, 0u);
            if (!is_e) {
                nph++;
                store_part(pq, bp + __popc(mp & lt), lx, ly, lz, P.u[i], P.v[i], P.w[i], P.E[i], (uint32_t)g,
                           (uint32_t)(g >> 32), 1u, pb);
            } else {
                nel++;
                if (local_e)
                    deposit<MODE>(T, A, voxel(T, lx, ly, lz), P.E[i], pb, 0u, 0u);
                else
                    enqueue_source_electron<MODE>(T, A, eq, be + __popc(me & lt), lx, ly, lz, P.u[i], P.v[i],
                                                  P.w[i], P.E[i], (uint32_t)g, (uint32_t)(g >> 32), pb);
            }
        }
    }
    esc = warp_sum(esc);
    const double dep = warp_sum(kval(A.dep) + (double)A.dep32);
    nph = warp_sum_u64(nph); nel = warp_sum_u64(nel); nmiss = warp_sum_u64(nmiss);
    if (lane == 0) {
        if (esc != 0.0) atomicAdd(&T.stats->ledger[2], esc);
        if (dep != 0.0) atomicAdd(&T.stats->ledger[3], dep);
        if (nph) atomicAdd(&T.stats->c[1], nph);
        if (nel) atomicAdd(&T.stats->c[2], nel);
        if (nmiss) atomicAdd(&T.stats->c[4], nmiss);
    }
}

// Philox key of the run, and a snapshot of the overflow counter taken in
// stream order (the host compares it with the counter after the run)
__global__ void k_set_key(uint32_t *key, uint32_t k0, uint32_t k1, const unsigned long long *ovf)
{
    key[0] = k0;
    key[1] = k1;
    *(unsigned long long *)(key + 2) = *ovf;
}

// ------------------------------------------------------ PSL-file source ---
// Particles read from PSL files (the comparator source model of Table 1):
// jaw test at the upper jaw surfaces, straight flight to the phantom surface,
// then the same compaction into the photon and electron queues as the
// sampler's. Record i of the chunk is history g0 + i and position i0 + i of
// the pass, which puts it in batch slot (i0 + i) mod nb. The test and the
// flight are written as single-precision roundings in a fixed order (no
// contraction), so that the accept and miss decisions are reproducible.
template <int MODE>
__global__ void __launch_bounds__(256) k_pslfile_enqueue(const PslRec *__restrict__ rec, int64_t n, uint64_t g0,
                                                         int64_t i0, int nb, PslGeom G, TP T, Queue pq, Queue eq)
{
    const unsigned lane = lane_id();
    unsigned lt;
    lanemask_lt(lt);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // source, rejected and missed energy per thread in FP64: the source
    // energy is the same sum, to FP64 rounding, however the run is split
    double src = 0.0, rej = 0.0, esc = 0.0;
    Acc A = {{0.0f, 0.0f}, {0.0f, 0.0f}, 0.0f, 0ull, 0ull, 0ull, 0ull};
    unsigned long long nph = 0, nel = 0, nrej = 0, nmiss = 0;
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const int64_t i = base + lane;
        bool in = false, is_e = false;
        float lx = 0.0f, ly = 0.0f, u = 0.0f, v = 0.0f, w = 1.0f, E = 0.0f;
        uint32_t tag = 0;
        if (i < n) {
            const float4 *r4 = reinterpret_cast<const float4 *>(rec + i);
            const float4 a = __ldg(r4), b = __ldg(r4 + 1);
            const float x = a.x, y = a.y;
            u = a.z; v = a.w; w = b.x; E = b.y;
            tag = __float_as_uint(b.z);
            is_e = (tag >> 16) == 1u;
            const float iw = __fdiv_rn(1.0f, w);
            const float yJ = __fadd_rn(y, __fmul_rn(__fmul_rn(G.zy_rel, v), iw));
            const float xJ = __fadd_rn(x, __fmul_rn(__fmul_rn(G.zx_rel, u), iw));
            src += E;
            if (!(yJ >= G.jaw[0] && yJ <= G.jaw[1] && xJ >= G.jaw[2] && xJ <= G.jaw[3])) {
                rej += E;
                nrej++;
            } else {
                lx = __fsub_rn(__fadd_rn(x, __fmul_rn(__fmul_rn(G.z_rel, u), iw)), G.x0);
                ly = __fsub_rn(__fadd_rn(y, __fmul_rn(__fmul_rn(G.z_rel, v), iw)), G.y0);
                in = voxel(T, lx, ly, 0.0f) >= 0;
                if (!in) { esc += E; nmiss++; }
            }
        }
        const bool local_e = in && is_e && T.electron_mode == 0;
        const unsigned mp = __ballot_sync(0xffffffffu, in && !is_e);
        const unsigned me = __ballot_sync(0xffffffffu, in && is_e && !local_e);
        uint32_t bp = 0, be = 0;
        if (lane == 0) {
            if (mp) bp = atomicAdd(&T.cnt->n[0], (uint32_t)__popc(mp));
            if (me) {
                be = atomicAdd(&T.cnt->n[2], (uint32_t)__popc(me));
                atomicAdd(&T.cnt->src_e, (uint32_t)__popc(me));
            }
        }
        bp = __shfl_sync(0xffffffffu, bp, 0);
        be = __shfl_sync(0xffffffffu, be, 0);
        if (in) {
            const uint64_t g = g0 + (uint64_t)i;
            const uint32_t pb = pb_make(tag & 0xFFFFu, 0u, (uint32_t)((i0 + i) % nb));
            if (!is_e) {
                nph++;
                store_part(pq, bp + __popc(mp & lt), lx, ly, 0.0f, u, v, w, E, (uint32_t)g, (uint32_t)(g >> 32), 1u,
                           pb);
            } else {
                nel++;
                if (local_e)
                    deposit<MODE>(T, A, voxel(T, lx, ly, 0.0f), E, pb, 0u, 0u);
                else
                    enqueue_source_electron<MODE>(T, A, eq, be + __popc(me & lt), lx, ly, 0.0f, u, v, w, E,
                                                  (uint32_t)g, (uint32_t)(g >> 32), pb);
            }
        }
    }
    const double src_d = warp_sum(src), rej_d = warp_sum(rej), esc_d = warp_sum(esc);
    const double dep = warp_sum(kval(A.dep) + (double)A.dep32);
    nph = warp_sum_u64(nph); nel = warp_sum_u64(nel); nrej = warp_sum_u64(nrej); nmiss = warp_sum_u64(nmiss);
    if (lane == 0) {
        atomicAdd(&T.stats->ledger[0], src_d);
        if (rej_d != 0.0) atomicAdd(&T.stats->ledger[1], rej_d);
        if (esc_d != 0.0) atomicAdd(&T.stats->ledger[2], esc_d);
        if (dep != 0.0) atomicAdd(&T.stats->ledger[3], dep);
        if (nph) atomicAdd(&T.stats->c[1], nph);
        if (nel) atomicAdd(&T.stats->c[2], nel);
        if (nrej) atomicAdd(&T.stats->c[3], nrej);
        if (nmiss) atomicAdd(&T.stats->c[4], nmiss);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&T.stats->c[0], (unsigned long long)n);
}

// ------------------------------------------------------------- tallies ---

__global__ void k_flush(float *__restrict__ part, double *__restrict__ batch, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n >> 2;
    float4 *p4 = reinterpret_cast<float4 *>(part);
    double2 *b2 = reinterpret_cast<double2 *>(batch);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 v = p4[i];
        if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f) {
            double2 a = b2[2 * i], b = b2[2 * i + 1];
            a.x += v.x; a.y += v.y; b.x += v.z; b.y += v.w;
            b2[2 * i] = a; b2[2 * i + 1] = b;
            p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = part[i];
        if (v != 0.0f) { batch[i] += v; part[i] = 0.0f; }
    }
}

// Iterations that hold k whole batches: fold each FP32 batch slice straight
// into the running sums and clear it.
// x + y = s + e exactly (Knuth's TwoSum; no operation may be contracted)
__device__ __forceinline__ void two_sum(float x, float y, float &s, float &e)
{
    s = __fadd_rn(x, y);
    const float yv = __fsub_rn(s, x);
    e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, yv)), __fsub_rn(y, yv));
}

// The slots' sum and sum of squares per cell, added to the FP64 totals. Each
// is accumulated in FP32 as a value and a running sum of the rounding errors
// of its additions (cascaded summation, Ogita, Rump & Oishi, SIAM J. Sci.
// Comput. 26, 2005), the squares split exactly into product and error by one
// FMA; the pair is converted to FP64 once per cell. The error relative to the
// sum of magnitudes is about (k 2^-24)^2, and a cell costs a few FP64
// operations instead of three per slot (this GPU's FP64 pipe is narrow).
__global__ void k_fold_slots(float *__restrict__ part, double *__restrict__ s1, double *__restrict__ s2,
                             int64_t ncell, int k)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += stride) {
        float a = 0.0f, ae = 0.0f, q2 = 0.0f, qe = 0.0f;
        bool any = false;
        for (int q = 0; q < k; ++q) {
            const float v = part[(size_t)q * ncell + c];
            if (v != 0.0f) {
                float t, e;
                two_sum(a, v, t, e);
                a = t;
                ae = __fadd_rn(ae, e);
                const float sq = __fmul_rn(v, v), sqe = __fmaf_rn(v, v, -sq);
                two_sum(q2, sq, t, e);
                q2 = t;
                qe = __fadd_rn(qe, __fadd_rn(e, sqe));
                part[(size_t)q * ncell + c] = 0.0f;
                any = true;
            }
        }
        if (any) {
            s1[c] += (double)a + (double)ae;
            s2[c] += (double)q2 + (double)qe;
        }
    }
}

__global__ void k_fold(double *__restrict__ batch, double *__restrict__ s1, double *__restrict__ s2, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = batch[i];
        if (v != 0.0) {
            s1[i] += v;
            s2[i] += v * v;
            batch[i] = 0.0;
        }
    }
}



// ---------------------------------------------------------- normalisation ---

// dose per source particle (MeV/g) and its batch standard deviation
// dose = S1 / B * scale / m and sigma = sqrt(B var) / B * scale / m, with
// var = max(S2 - S1^2 / B, 0) / (B - 1) the batch variance and m = rho V;
// written as dose = S1 f_d / m, sigma = sqrt(max(S2 - S1^2 / B, 0) f_v) scale / m
// (f_d = scale / B, f_v = 1 / (B (B - 1)), 0 for B = 1) with 1 / m stored per
// voxel, so that a voxel costs one FP64 square root and no division
__global__ void k_dose(const double *__restrict__ s1, const double *__restrict__ s2,
                       const double *__restrict__ inv_mass, int64_t n, double inv_b, double f_d, double f_v,
                       double scale, double *__restrict__ dose, double *__restrict__ sigma)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double im = inv_mass[i];
        const double a = s1[i];
        dose[i] = a * f_d * im;
        if (sigma) sigma[i] = sqrt(fmax(s2[i] - a * a * inv_b, 0.0) * f_v) * scale * im;
    }
}

// A[(b,row),k] = S1 / B * scale(k,b) / (rho V of the row's voxel)
__global__ void k_basis(const double *__restrict__ s1, const double *__restrict__ cell_scale,
                        const double *__restrict__ row_mass, int n_rows, int n_psr, int n_beams, int B,
                        double *__restrict__ A)
{
    const int64_t n = (int64_t)n_beams * n_rows * n_psr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int k = (int)(i % n_psr);
        const int64_t br = i / n_psr;
        const int row = (int)(br % n_rows), b = (int)(br / n_rows);
        const double m = row_mass[row];
        A[i] = m > 0.0 ? s1[i] / B * cell_scale[(size_t)k * n_beams + b] / m : 0.0;
    }
}

// The same matrix with the electron PSRs of each energy bin summed into one
// column (the effective electron unit of Sec. 2.2.3): columns [0, n_ph) are
// the photon PSRs, column n_ph + e the n_r electron PSRs of bin e added in
// ring order.
__global__ void k_basis_units(const double *__restrict__ s1, const double *__restrict__ cell_scale,
                              const double *__restrict__ row_mass, int n_rows, int n_psr, int n_ph, int n_r,
                              int n_beams, int B, double *__restrict__ A)
{
    const int n_col = n_ph + (n_psr - n_ph) / n_r;
    const int64_t n = (int64_t)n_beams * n_rows * n_col;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int j = (int)(i % n_col);
        const int64_t br = i / n_col;
        const int row = (int)(br % n_rows), b = (int)(br / n_rows);
        const double m = row_mass[row];
        const double *s = s1 + br * n_psr;
        double v = 0.0;
        if (m > 0.0) {
            if (j < n_ph) {
                v = s[j] / B * cell_scale[(size_t)j * n_beams + b] / m;
            } else {
                const int k0 = n_ph + (j - n_ph) * n_r;
                for (int R = 0; R < n_r; ++R) v += s[k0 + R] / B * cell_scale[(size_t)(k0 + R) * n_beams + b] / m;
            }
        }
        A[i] = v;
    }
}

// per (PSR, beam) scale of a per-PSR plan, gathered from the entry table
__global__ void k_cell_scale(const EntryRec *__restrict__ ent, const double *__restrict__ escale, int64_t n_ent,
                             int n_e, int n_r, int n_beams, double *__restrict__ cell_scale)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_ent) return;
    const EntryRec e = ent[i];
    const int k = ((int)e.stype * n_e + e.ebin) * n_r + e.fixed_ring;
    cell_scale[(size_t)k * n_beams + e.beam] = escale[i];   // identical for every entry of (k, b)
}

// mass of the voxel each basis row refers to
__global__ void k_row_mass(const uint16_t *__restrict__ idx, const float *__restrict__ rho, int64_t nvox,
                           int n_rows, double vol, double *__restrict__ row_mass)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
        const int r = idx[i];
        if (r && r <= n_rows) row_mass[r - 1] = (double)rho[i] * vol;
    }
}

// ------------------------------------------------------------ host side ---

// polls of a transport CTA's table-staging wait (lsm_set_wait_limits)
int g_stage_polls = 1 << 22;

lsm_status read_fallbacks(int64_t *count, int reset)
{
    unsigned long long v = 0;
    LSM_CUDA(cudaDeviceSynchronize());
    LSM_CUDA(cudaMemcpyFromSymbol(&v, g_stage_fallbacks, sizeof(v)));
    if (count) *count = (int64_t)v;
    if (reset) {
        v = 0;
        LSM_CUDA(cudaMemcpyToSymbol(g_stage_fallbacks, &v, sizeof(v)));
    }
    return LSM_OK;
}

namespace {

int grid_for(const void *fn, int threads, size_t smem)
{
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
    if (per < 1) per = 1;
    return per * sm_count();
}

struct Workspace {
    Queue q[3];          // 0 primary photons, 2 electrons (1 is empty: annihilation photons are
                         // tracked by the lane of their pair event)
    IterCounters *cnt;
    uint32_t *key;       // Philox key of the run (outside the per-iteration counters)
    void *mem;
};

// Queues live in one allocation cached on the tally and reused by later runs
// (a second one for the second half-iteration of two-stream runs).
cudaError_t ws_alloc_at(Workspace &W, uint32_t chunk, uint32_t ecap, void *&mem, uint32_t &mem_chunk,
                        uint32_t &mem_ecap, cudaStream_t st)
{
    if (mem && mem_chunk >= chunk && mem_ecap >= ecap) {
        chunk = mem_chunk;
        ecap = mem_ecap;
    } else {
        if (mem) cudaFreeAsync(mem, st);
        mem = nullptr;
        size_t total = 2048;
        const uint32_t c2[3] = {chunk, 0, ecap};
        for (int k = 0; k < 3; ++k) total += (size_t)c2[k] * 48 + 256;
        cudaError_t e = dev_malloc(&mem, total, st);
        if (e != cudaSuccess) return e;
        mem_chunk = chunk;
        mem_ecap = ecap;
    }
    const uint32_t caps[3] = {chunk, 0, ecap};
    char *p = (char *)mem;
    W.mem = nullptr;
    static_assert(sizeof(IterCounters) <= 1024, "iteration counters overlap the key");
    W.cnt = (IterCounters *)p;
    W.key = (uint32_t *)(p + 1024);
    p += 2048;
    for (int k = 0; k < 3; ++k) {
        Queue &q = W.q[k];
        q.cap = caps[k];
        q.rec = (float4 *)p;
        p += ((size_t)caps[k] * 48 + 255) / 256 * 256;
    }
    return cudaSuccess;
}

cudaError_t ws_alloc(Workspace &W, uint32_t chunk, uint32_t ecap, lsm_tally *t, cudaStream_t st)
{
    return ws_alloc_at(W, chunk, ecap, t->ws, t->ws_chunk, t->ws_ecap, st);
}

// A run's secondary-electron queue capacity: the workspace's, or less when
// the run asks for a smaller queue (e_queue_cap).
void cap_equeue(Workspace &W, const lsm_run_opts &o)
{
    if (o.e_queue_cap > 0 && (uint32_t)o.e_queue_cap < W.q[2].cap) W.q[2].cap = (uint32_t)o.e_queue_cap;
}

TP make_tp(const lsm_phantom *ph, const lsm_tally *t, const lsm_run_opts &o, const uint32_t *key, IterCounters *cnt)
{
    TP T;
    T.hl = t->hl;
    T.hl_g0 = t->hl_g0;
    T.hl_n = t->hl_n;
    T.rhomat = ph->d_rhomat;
    T.nx = ph->nx; T.ny = ph->ny; T.nz = ph->nz;
    T.inv_dx = (float)(1.0 / ph->dx); T.inv_dy = (float)(1.0 / ph->dy); T.inv_dz = (float)(1.0 / ph->dz);
    T.lx = (float)(ph->nx * ph->dx); T.ly = (float)(ph->ny * ph->dy);
    T.xs = ph->d_xs; T.mumax = ph->d_mumax;
    T.inv_dlnE = (float)((kGrid - 1) / (kLnEmax - kLnEmin));
    T.maj = (float)o.majorant_factor;
    T.part = t->d_part;
    T.ncell = t->ncell;
    T.idx = t->mode == 1 ? t->d_idx : nullptr;
    T.n_rows = t->n_rows; T.n_psr = t->n_psr; T.n_beams = t->n_beams;
    T.electron_mode = o.electron_mode;
    T.max_steps = o.max_steps;
    T.f_e = (float)o.f_e;
    const double sg = o.s_geo > 0 ? o.s_geo : 0.5 * fmin(ph->dx, fmin(ph->dy, ph->dz));
    T.s_geo = (float)sg;
    T.key = key;
    T.ph_bad = ph->d_flags + 2;
    T.ctas_per_sm = o.ctas_per_sm;
    T.stage_polls = g_stage_polls;
    T.stats = t->d_stats;
    T.cnt = cnt;
    return T;
}

lsm_status check_opts(lsm_run_opts &o)
{
    if (o.ctas_per_sm < 0) return set_arg_error("ctas_per_sm must be >= 0");
    if (o.electron_mode != 0 && o.electron_mode != 1) return set_arg_error("electron_mode must be 0 or 1");
    if (!(o.majorant_factor >= 1.0) || !isfinite(o.majorant_factor)) return set_arg_error("majorant_factor must be >= 1");
    if (!(o.f_e > 0.0 && o.f_e <= 1.0)) return set_arg_error("f_e must be in (0, 1]");
    if (o.max_steps < 1) return set_arg_error("max_steps must be >= 1");
    if (o.chunk <= 0) o.chunk = 1 << 23;
    if (o.chunk > (1 << 24)) return set_arg_error("chunk must be <= 2^24");
    if (o.n_batches < 1) o.n_batches = 1;
    if (o.first_batch < 0) return set_arg_error("first_batch must be >= 0");
    if (o.e_queue_cap < 0) return set_arg_error("e_queue_cap must be >= 0");
    if (o.streams == 0) o.streams = 1;
    if (o.streams != 1 && o.streams != 2) return set_arg_error("streams must be 1 or 2");
    return LSM_OK;
}

// transport everything queued in W (photons of queue 0 with the annihilation
// photons they create, then electrons)
template <int MODE>
lsm_status drain(const TP &T, Workspace &W, lsm_tally *t, cudaStream_t st)
{
    const size_t smem = (size_t)kTableBytes, smem_e = (size_t)kXsBytes;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_transport<MODE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_transport<MODE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e);
        attr = true;
    }
    static int gp_max = 0, ge_max = 0;
    if (!gp_max) gp_max = grid_for((const void *)k_transport<MODE, 0>, LSM_PHOTON_THREADS, smem);
    if (!ge_max) ge_max = grid_for((const void *)k_transport<MODE, 1>, LSM_ELECTRON_THREADS, smem_e);
    const int cap = T.ctas_per_sm > 0 ? T.ctas_per_sm * sm_count() : (1 << 30);
    const int gp = std::min(gp_max, cap), ge = std::min(ge_max, cap);
    int tk = timer_begin(2, st);
    k_transport<MODE, 0><<<gp, LSM_PHOTON_THREADS, smem, st>>>(T, W.q[0], 0, W.q[2]);
    LSM_LAUNCHED("k_transport<photon>");
    timer_end(tk, st);
    if (T.electron_mode) {
        tk = timer_begin(4, st);
        k_transport<MODE, 1><<<ge, LSM_ELECTRON_THREADS, smem_e, st>>>(T, W.q[2], 2, W.q[2]);
        LSM_LAUNCHED("k_transport<electron>");
        timer_end(tk, st);
    }
    return LSM_OK;
}

// queue overflows (run statistics counter 9) since k_set_key; synchronises
lsm_status read_overflow(lsm_tally *t, const Workspace &W, cudaStream_t st, unsigned long long *out)
{
    unsigned long long v[2] = {0, 0};
    LSM_CUDA(cudaMemcpyAsync(&v[0], &t->d_stats->c[9], 8, cudaMemcpyDeviceToHost, st));
    LSM_CUDA(cudaMemcpyAsync(&v[1], W.key + 2, 8, cudaMemcpyDeviceToHost, st));
    LSM_CUDA(cudaStreamSynchronize(st));
    *out = v[0] - v[1];
    return LSM_OK;
}

void set_key(const Workspace &W, lsm_tally *t, uint64_t seed, cudaStream_t st)
{
    k_set_key<<<1, 1, 0, st>>>(W.key, (uint32_t)seed, (uint32_t)(seed >> 32), &t->d_stats->c[9]);
    count_launch();
}

}  // namespace

lsm_status fold_batch(lsm_tally *t, cudaStream_t st, bool count)
{
    const int64_t n = t->ncell;
    const int g = (int)std::min<int64_t>((n + 255) / 256, 8 * sm_count());
    const int tk = timer_begin(5, st);
    k_fold<<<g, 256, 0, st>>>(t->d_batch, t->d_s1, t->d_s2, n);
    count_launch();
    timer_end(tk, st);
    LSM_CUDA(cudaGetLastError());
    if (count) t->n_batches++;
    return LSM_OK;
}

lsm_status flush_partials(lsm_tally *t, cudaStream_t st)
{
    const int64_t n = t->ncell;
    const int gf = (int)std::min<int64_t>((n / 4 + 255) / 256 + 1, 8 * sm_count());
    const int tk = timer_begin(5, st);
    k_flush<<<gf, 256, 0, st>>>(t->d_part, t->d_batch, n);
    count_launch();
    timer_end(tk, st);
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

// fold k whole-batch slices of the partial tally into S1/S2
lsm_status fold_slots(lsm_tally *t, int k, cudaStream_t st)
{   // batches are counted by the caller
    const int64_t n = t->ncell;
    const int g = (int)std::min<int64_t>((n + 255) / 256, 8 * sm_count());
    const int tk = timer_begin(5, st);
    k_fold_slots<<<g, 256, 0, st>>>(t->d_part, t->d_s1, t->d_s2, n, k);
    count_launch();
    timer_end(tk, st);
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

// make room for `slots` partial-tally slices (pending slot-0 partials are flushed first)
lsm_status ensure_slots(lsm_tally *t, int slots, cudaStream_t st)
{
    if (slots <= t->part_slots) return LSM_OK;
    lsm_status rc = flush_partials(t, st);
    if (rc) return rc;
    float *np = nullptr;
    LSM_CUDA(dev_malloc((void **)&np, (size_t)slots * t->ncell * 4 + 16, st));
    LSM_CUDA(cudaMemsetAsync(np, 0, (size_t)slots * t->ncell * 4, st));
    LSM_CUDA(cudaFreeAsync(t->d_part, st));
    t->d_part = np;
    t->part_slots = slots;
    return LSM_OK;
}

lsm_status resolve_psl(lsm_psl *P);

lsm_status sample_public(const lsm_psl *P, uint64_t seed, uint64_t g0, int64_t n, double z_surf,
                         const lsm_particles *out, cudaStream_t st)
{
    if (!P || !out) return set_arg_error("lsm_sample: NULL argument");
    {
        const lsm_status r = resolve_psl(const_cast<lsm_psl *>(P));
        if (r) return r;
    }
    if (n < 0) return set_arg_error("lsm_sample: n < 0");
    if (n == 0) return LSM_OK;
    if (!out->x || !out->y || !out->z || !out->u || !out->v || !out->w || !out->E || !out->hist || !out->psr ||
        !out->beam || !out->type || !out->status)
        return set_arg_error("lsm_sample: NULL output array");
    const int64_t h0 = (int64_t)(g0 % (uint64_t)P->plan_size);
    const int g = (int)std::min<int64_t>((n + 255) / 256, 16 * sm_count());
    k_sample_public<<<g, 256, 0, st>>>(P->sp, (uint32_t)seed, (uint32_t)(seed >> 32), g0, h0, P->plan_size, n,
                                       (float)(z_surf - P->z_phsp), (float)z_surf, *out);
    LSM_LAUNCHED("k_sample_public");
    return LSM_OK;
}

lsm_status transport_particles(const lsm_phantom *ph, const lsm_particles *in, int64_t n, uint64_t seed,
                               lsm_tally *t, const lsm_run_opts *opts, cudaStream_t st)
{
    if (!ph || !in || !t || !opts) return set_arg_error("lsm_transport: NULL argument");
    if (n < 0 || n > (1 << 24)) return set_arg_error("lsm_transport: 0 <= n <= 2^24");
    lsm_run_opts o = *opts;
    lsm_status rc = check_opts(o);
    if (rc) return rc;
    if (t->nvox != (int64_t)ph->nx * ph->ny * ph->nz) return set_arg_error("lsm_transport: tally of another phantom");
    if (n == 0) return LSM_OK;
    Workspace W = {};
    const uint32_t cap = (uint32_t)std::max<int64_t>(n, 1024);
    unsigned long long ovf = 0;
    cudaError_t e = ws_alloc(W, cap, (uint32_t)std::min<int64_t>(8 * (int64_t)cap + (1 << 18), 1u << 28), t, st);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_transport workspace");
    cap_equeue(W, o);
    TP T = make_tp(ph, t, o, W.key, W.cnt);
    do {
        set_key(W, t, seed, st);
        if ((e = cudaMemsetAsync(W.cnt, 0, sizeof(IterCounters), st)) != cudaSuccess) { rc = set_cuda_error(e, "memset"); break; }
        const int g = (int)std::min<int64_t>((n + 255) / 256, 8 * sm_count());
        if (t->mode == 0)
            k_enqueue<0><<<g, 256, 0, st>>>(*in, n, (float)ph->x0, (float)ph->y0, (float)ph->z0, T, W.q[0], W.q[2]);
        else
            k_enqueue<1><<<g, 256, 0, st>>>(*in, n, (float)ph->x0, (float)ph->y0, (float)ph->z0, T, W.q[0], W.q[2]);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) { rc = set_cuda_error(e, "k_enqueue"); break; }
        rc = t->mode == 0 ? drain<0>(T, W, t, st) : drain<1>(T, W, t, st);
        if (rc) break;
        rc = flush_partials(t, st);
        if (rc) break;
        rc = read_overflow(t, W, st, &ovf);
    } while (0);
    if (rc) return rc;
    if (ovf) return LSM_ERR_OVERFLOW;
    return LSM_OK;
}

// PSL-file runs: one workspace for the whole run; every chunk of records is
// enqueued and transported in stream order without host synchronisation, its
// deposits landing in the batch slot of each record; a pass ends by folding
// the nb slots into S1/S2 as nb batches.
struct PslFileRun {
    Workspace W;
    TP T;
    lsm_tally *t;
    int nb;
};

lsm_status pslfile_begin(const lsm_phantom *ph, lsm_tally *t, const lsm_run_opts *opts, int64_t cap, int nb,
                         uint64_t seed, cudaStream_t st, PslFileRun **out)
{
    *out = nullptr;
    if (t->nvox != (int64_t)ph->nx * ph->ny * ph->nz) return set_arg_error("lsm_pslfile_run: tally of another phantom");
    if (t->mode != 0) return set_arg_error("lsm_pslfile_run: needs a dose (mode 0) tally");
    if (nb < 1 || nb > 255) return set_arg_error("lsm_pslfile_run: 1 <= n_batches <= 255");
    if (cap < 1 || cap > (1 << 24)) return set_arg_error("lsm_pslfile_run: 1 <= chunk <= 2^24");
    lsm_run_opts o = *opts;
    lsm_status rc = check_opts(o);
    if (rc) return rc;
    rc = ensure_slots(t, nb, st);
    if (rc) return rc;
    PslFileRun *R = new PslFileRun();
    const uint32_t c = (uint32_t)std::max<int64_t>(cap, 1024);
    cudaError_t e = ws_alloc(R->W, c, (uint32_t)std::min<int64_t>(4 * (int64_t)c + (1 << 18), 0xF0000000ll), t, st);
    if (e != cudaSuccess) { delete R; return set_cuda_error(e, "lsm_pslfile_run workspace"); }
    cap_equeue(R->W, o);
    R->T = make_tp(ph, t, o, R->W.key, R->W.cnt);
    R->t = t;
    R->nb = nb;
    set_key(R->W, t, seed, st);
    *out = R;
    return LSM_OK;
}

lsm_status pslfile_chunk(PslFileRun *R, const void *d_rec, int64_t n, uint64_t g0, int64_t i0, const PslGeom &G,
                         cudaStream_t st)
{
    if (n <= 0) return LSM_OK;
    if (n > (int64_t)R->W.q[0].cap) return set_arg_error("lsm_pslfile_run: chunk larger than the workspace");
    LSM_CUDA(cudaMemsetAsync(R->W.cnt, 0, sizeof(IterCounters), st));
    const int g = (int)std::min<int64_t>((n + 255) / 256, 8 * sm_count());
    const int tk = timer_begin(1, st);
    k_pslfile_enqueue<0><<<g, 256, 0, st>>>((const PslRec *)d_rec, n, g0, i0, R->nb, G, R->T, R->W.q[0], R->W.q[2]);
    count_launch();
    timer_end(tk, st);
    LSM_CUDA(cudaGetLastError());
    return drain<0>(R->T, R->W, R->t, st);
}

lsm_status pslfile_end_pass(PslFileRun *R, cudaStream_t st)
{
    lsm_status rc = fold_slots(R->t, R->nb, st);
    if (rc == LSM_OK) R->t->n_batches += R->nb;
    return rc;
}

// releases the run; returns LSM_ERR_OVERFLOW if a queue filled up (synchronises)
lsm_status pslfile_finish(PslFileRun *R, cudaStream_t st)
{
    if (!R) return LSM_OK;
    unsigned long long ovf = 0;
    lsm_status rc = read_overflow(R->t, R->W, st, &ovf);
    delete R;
    if (rc) return rc;
    return ovf ? LSM_ERR_OVERFLOW : LSM_OK;
}

lsm_status run_plan(const lsm_psl *P, const lsm_phantom *ph, lsm_tally *t, uint64_t seed,
                    const lsm_run_opts *opts, cudaStream_t st)
{
    if (!P || !ph || !t || !opts) return set_arg_error("lsm_run: NULL argument");
    lsm_run_opts o = *opts;
    lsm_status rc = check_opts(o);
    if (rc) return rc;
    if (t->nvox != (int64_t)ph->nx * ph->ny * ph->nz) return set_arg_error("lsm_run: tally of another phantom");
    if (t->mode == 1 && (t->n_beams != P->n_beams || t->n_psr != 3 * P->n_e * P->n_r))
        return set_arg_error("lsm_run: basis tally shape does not match the plan");
    // a per-history energy ledger (test mode) selects the MODE 2 kernels, run
    // directly (a captured graph holds the kernels of one mode)
    const int kmode = t->mode == 1 ? 1 : (t->hl ? 2 : 0);
    if (t->hl) o.use_graph = 0;
    // Iteration size. The paper iterates M histories at a time (Sec. 2.1.3);
    // B300 keeps ~2e5 lanes resident, so an iteration should hold millions of
    // histories for its longest tracks not to dominate. Plans smaller than
    // the iteration size are run k whole batches per iteration, each batch in
    // its own slice of the partial tally; larger plans are split into
    // iterations inside one batch.
    const int64_t plan = P->plan_size;
    const bool multi = plan < (int64_t)o.chunk;
    // (at most 255 batches per iteration: a particle carries its batch slot in
    // 8 bits; more batches take more iterations)
    const int bpi = multi ? (int)std::min<int64_t>(std::min<int64_t>(o.n_batches, 255), (int64_t)o.chunk / plan) : 1;
    const int64_t chunk = multi ? (int64_t)bpi * plan : (int64_t)o.chunk;
    Workspace W = {};
    unsigned long long ovf = 0;
    rc = ensure_slots(t, bpi, st);
    if (rc) return rc;
    cudaError_t e = ws_alloc(W, (uint32_t)chunk, (uint32_t)std::min<int64_t>(4 * chunk + (1 << 18), 0xF0000000ll), t, st);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_run workspace");
    cap_equeue(W, o);
    TP T = make_tp(ph, t, o, W.key, W.cnt);
    SQ S;
    S.sp = P->sp;
    S.key = W.key;
    S.z_rel = (float)(ph->z0 - P->z_phsp);
    S.x0 = (float)ph->x0; S.y0 = (float)ph->y0;
    S.z0 = (float)ph->z0; S.lz = (float)(ph->nz * ph->dz);
    S.plan = plan;
    static int gs0 = 0, gs1 = 0, gs2 = 0;
    if (!gs0) gs0 = grid_for((const void *)k_sample_queue<0>, 256, 0);
    if (!gs1) gs1 = grid_for((const void *)k_sample_queue<1>, 256, 0);
    if (!gs2) gs2 = grid_for((const void *)k_sample_queue<2>, 256, 0);
    // Two-stream runs (streams = 2, several batches per iteration): each
    // iteration's batches are split into two halves with their own queues,
    // sampled and transported on two streams, so that each half's passes
    // fill the SMs the other half's passes leave idle at the end of their
    // queues; the halves tally into different batch slots, and the slots are
    // folded once both are done.
    const bool two = o.streams == 2 && multi && bpi >= 2;
    Workspace W2 = {};
    TP T2 = T;
    SQ S2 = S;
    cudaStream_t s2 = nullptr;
    if (two) {
        const int64_t half = (int64_t)((bpi + 1) / 2) * plan;
        e = ws_alloc_at(W2, (uint32_t)half, (uint32_t)std::min<int64_t>(4 * half + (1 << 18), 0xF0000000ll), t->ws2,
                        t->ws2_chunk, t->ws2_ecap, st);
        if (e != cudaSuccess) return set_cuda_error(e, "lsm_run second workspace");
        cap_equeue(W2, o);
        T2 = make_tp(ph, t, o, W2.key, W2.cnt);
        S2.key = W2.key;
        if (!t->pstream) {
            cudaStream_t ps = nullptr;
            LSM_CUDA(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
            cudaEvent_t e1 = nullptr, e2 = nullptr;
            LSM_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
            LSM_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
            t->pstream = ps; t->pev[0] = e1; t->pev[1] = e2;
        }
        s2 = (cudaStream_t)t->pstream;
    }
    auto iteration_on = [&](Workspace &Wx, const TP &Tx, SQ &Sx, cudaStream_t sx, uint64_t g0, int64_t h0,
                            int64_t n) -> lsm_status {
        Sx.g0 = g0;
        Sx.h0 = h0;
        Sx.n = n;
        LSM_CUDA(cudaMemsetAsync(Wx.cnt, 0, sizeof(IterCounters), sx));
        const int gs = (int)std::min<int64_t>((Sx.n + 255) / 256, kmode == 0 ? gs0 : (kmode == 1 ? gs1 : gs2));
        const int tk = timer_begin(1, sx);
        if (kmode == 0) k_sample_queue<0><<<gs, 256, 0, sx>>>(Sx, Tx, Wx.q[0], Wx.q[2]);
        else if (kmode == 1) k_sample_queue<1><<<gs, 256, 0, sx>>>(Sx, Tx, Wx.q[0], Wx.q[2]);
        else k_sample_queue<2><<<gs, 256, 0, sx>>>(Sx, Tx, Wx.q[0], Wx.q[2]);
        count_launch();
        timer_end(tk, sx);
        LSM_CUDA(cudaGetLastError());
        return kmode == 0 ? drain<0>(Tx, Wx, t, sx) : (kmode == 1 ? drain<1>(Tx, Wx, t, sx) : drain<2>(Tx, Wx, t, sx));
    };
    auto iteration = [&](uint64_t g0, int64_t h0, int64_t n) -> lsm_status {
        return iteration_on(W, T, S, st, g0, h0, n);
    };
    // the whole run's launch sequence (no host synchronisation inside)
    auto enqueue = [&]() -> lsm_status {
        lsm_status r = LSM_OK;
        if (multi) {
            for (int b0 = 0; b0 < o.n_batches && r == LSM_OK; b0 += bpi) {
                const int k = std::min(bpi, o.n_batches - b0);
                const uint64_t g0 = (uint64_t)(o.first_batch + b0) * (uint64_t)plan;
                if (two && k >= 2) {
                    const int ka = (k + 1) / 2;
                    LSM_CUDA(cudaEventRecord((cudaEvent_t)t->pev[0], st));
                    LSM_CUDA(cudaStreamWaitEvent(s2, (cudaEvent_t)t->pev[0], 0));
                    r = iteration_on(W, T, S, st, g0, 0, (int64_t)ka * plan);
                    if (r == LSM_OK)
                        r = iteration_on(W2, T2, S2, s2, g0 + (uint64_t)ka * plan, (int64_t)ka * plan,
                                         (int64_t)(k - ka) * plan);
                    LSM_CUDA(cudaEventRecord((cudaEvent_t)t->pev[1], s2));
                    LSM_CUDA(cudaStreamWaitEvent(st, (cudaEvent_t)t->pev[1], 0));
                } else {
                    r = iteration(g0, 0, (int64_t)k * plan);
                }
                if (r == LSM_OK) r = fold_slots(t, k, st);
            }
        } else {
            for (int b = 0; b < o.n_batches && r == LSM_OK; ++b) {
                for (int64_t h0 = 0; h0 < plan && r == LSM_OK; h0 += chunk) {
                    r = iteration((uint64_t)(o.first_batch + b) * (uint64_t)plan + (uint64_t)h0, h0,
                                  std::min<int64_t>(chunk, plan - h0));
                    if (r == LSM_OK) r = flush_partials(t, st);
                }
                if (r == LSM_OK) r = fold_batch(t, st, false);
            }
        }
        return r;
    };
    set_key(W, t, seed, st);
    if (two) set_key(W2, t, seed, st);
    LSM_CUDA(cudaGetLastError());
    bool replayed = false;
    if (o.use_graph) {
        // One CUDA graph per (plan, phantom, tally buffers, options): captured
        // on first use, replayed afterwards with only the key set outside it.
        // Capture and replay use the tally's own stream (the legacy default
        // stream cannot be captured), ordered against `st` by events.
        if (!t->gstream) {
            cudaStream_t gs = nullptr;
            LSM_CUDA(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
            cudaEvent_t e1 = nullptr, e2 = nullptr;
            LSM_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
            LSM_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
            t->gstream = gs; t->gev[0] = e1; t->gev[1] = e2;
        }
        const cudaStream_t caller = st;
        st = (cudaStream_t)t->gstream;
        LSM_CUDA(cudaEventRecord((cudaEvent_t)t->gev[0], caller));
        LSM_CUDA(cudaStreamWaitEvent(st, (cudaEvent_t)t->gev[0], 0));
        GraphKey gk;
        memset(&gk, 0, sizeof(GraphKey));
        gk.timed = timing_enabled() ? 1 : 0;
        gk.psl = P->uid; gk.ph = ph->uid; gk.part = t->d_part; gk.ws = t->ws; gk.batch = t->d_batch;
        gk.ws2 = t->ws2;
        gk.o = o;
        gk.o.n_batches = o.n_batches;
        if (!t->gexec || memcmp(&gk, &t->gkey, sizeof(GraphKey)) != 0) {
            memset(&t->gkey, 0, sizeof(GraphKey));
            if (t->gexec) { cudaGraphExecDestroy((cudaGraphExec_t)t->gexec); t->gexec = nullptr; }
            timer_free(t->gtimers);
            t->gtimers = nullptr;
            const int64_t l0 = lsm_launch_count();
            const size_t tm0 = timer_mark();
            LSM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            rc = enqueue();
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(st, &g);
            void *tset = timer_detach(tm0);
            if (rc == LSM_OK && ce != cudaSuccess) rc = set_cuda_error(ce, "lsm_run: graph capture");
            if (rc == LSM_OK) {
                cudaGraphExec_t ge = nullptr;
                ce = cudaGraphInstantiate(&ge, g, 0);
                if (ce != cudaSuccess) rc = set_cuda_error(ce, "lsm_run: graph instantiate");
                else {
                    t->gexec = ge;
                    memcpy(&t->gkey, &gk, sizeof(GraphKey));
                    t->graph_kernels = lsm_launch_count() - l0;
                    t->gtimers = tset;
                    tset = nullptr;
                }
            }
            timer_free(tset);
            if (g) cudaGraphDestroy(g);
            if (rc) return rc;
        } else {
            add_launches(t->graph_kernels);
        }
        LSM_CUDA(cudaGraphLaunch((cudaGraphExec_t)t->gexec, st));
        replayed = true;
        LSM_CUDA(cudaEventRecord((cudaEvent_t)t->gev[1], st));
        LSM_CUDA(cudaStreamWaitEvent(caller, (cudaEvent_t)t->gev[1], 0));
        st = caller;
    } else {
        rc = enqueue();
        if (rc) return rc;
    }
    t->n_batches += o.n_batches;
    if (o.no_sync) {                        // overflows stay counted in the run statistics
        if (replayed && t->gtimers) {       // a replay's timer events are read once complete
            LSM_CUDA(cudaStreamSynchronize(st));
            timer_replayed(t->gtimers);
        }
        return LSM_OK;
    }
    rc = read_overflow(t, W, st, &ovf);
    if (rc) return rc;
    if (replayed) timer_replayed(t->gtimers);
    rc = resolve_psl(const_cast<lsm_psl *>(P));
    if (rc) return rc;
    if (ovf) return LSM_ERR_OVERFLOW;
    return LSM_OK;
}

lsm_status dose_impl(const lsm_tally *t, const lsm_phantom *ph, double scale, double *dose, double *sigma,
                     lsm_mem mem, cudaStream_t st)
{
    if (!t || !ph || !dose) return set_arg_error("lsm_dose: NULL argument");
    if (t->mode != 0) return set_arg_error("lsm_dose: needs an energy (mode 0) tally");
    if (t->n_batches < 1) return set_arg_error("lsm_dose: no batch folded yet");
    const int64_t n = t->nvox;
    double *dd = dose, *ds = sigma;
    void *tmp = nullptr;
    unsigned bad = 0;
    if (mem == LSM_MEM_HOST) {
        LSM_CUDA(dev_malloc(&tmp, (size_t)n * 16, st));
        dd = (double *)tmp;
        ds = sigma ? dd + n : nullptr;
    }
    const int g = (int)std::min<int64_t>((n + 255) / 256, 8 * sm_count());
    const int B = t->n_batches;
    k_dose<<<g, 256, 0, st>>>(t->d_s1, t->d_s2, ph->d_inv_mass, n, 1.0 / B, scale / B,
                              B > 1 ? 1.0 / ((double)B * (B - 1)) : 0.0, scale, dd, ds);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem == LSM_MEM_HOST) {
        e = cudaMemcpyAsync(dose, dd, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && sigma) e = cudaMemcpyAsync(sigma, ds, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
        // a phantom created without the host check: its verdict comes back too
        if (e == cudaSuccess && !ph->validated)
            e = cudaMemcpyAsync(&bad, ph->d_flags + 2, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (tmp) cudaFreeAsync(tmp, st);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_dose");
    if (bad) return set_arg_error("lsm_dose: the phantom's densities must be in [1e-4, 25] and materials in {0, 1}");
    return LSM_OK;
}

lsm_status basis_impl(const lsm_tally *t, const lsm_psl *P, const lsm_phantom *ph, const uint16_t *idx3d,
                      lsm_mem idx_mem, double *A, lsm_mem mem, cudaStream_t st, bool units)
{
    if (!t || !P || !ph || !A) return set_arg_error("lsm_basis_matrix: NULL argument");
    if (units && t->n_psr != 3 * P->n_e * P->n_r)
        return set_arg_error("lsm_basis_matrix_units: the tally's PSR count must be 3 n_e n_r of the plan");
    if (t->mode != 1 || !P->per_psr) return set_arg_error("lsm_basis_matrix: needs a basis tally and a per-PSR plan");
    {
        const lsm_status r = resolve_psl(const_cast<lsm_psl *>(P));
        if (r) return r;
    }
    if (t->n_batches < 1) return set_arg_error("lsm_basis_matrix: no batch folded yet");
    const int npsr = t->n_psr, nb = t->n_beams, nr = t->n_rows;
    const int n_ph = 2 * P->n_e * P->n_r, n_col = units ? n_ph + P->n_e : npsr;
    const int64_t ncell = (int64_t)nb * nr * n_col;
    char *tmp = nullptr;
    const size_t bytes = (size_t)npsr * nb * 8 + (size_t)nr * 8 + (mem == LSM_MEM_HOST ? (size_t)ncell * 8 : 0) + 64;
    LSM_CUDA(dev_malloc((void **)&tmp, bytes, st));
    double *cs = (double *)tmp, *rm = cs + (size_t)npsr * nb;
    double *dA = mem == LSM_MEM_HOST ? rm + nr : A;
    cudaError_t e = cudaMemsetAsync(tmp, 0, (size_t)npsr * nb * 8 + (size_t)nr * 8, st);
    const uint16_t *didx = t->d_idx;
    (void)idx3d; (void)idx_mem;
    if (e == cudaSuccess) {
        k_cell_scale<<<(unsigned)((P->n_ent + 255) / 256), 256, 0, st>>>(P->d_ent, P->d_escale, P->n_ent, P->n_e,
                                                                          P->n_r, nb, cs);
        count_launch();
        const int g = (int)std::min<int64_t>((t->nvox + 255) / 256, 8 * sm_count());
        k_row_mass<<<g, 256, 0, st>>>(didx, ph->d_rho, t->nvox, nr, ph->dx * ph->dy * ph->dz, rm);
        count_launch();
        const int g2 = (int)std::min<int64_t>((ncell + 255) / 256, 8 * sm_count());
        if (units)
            k_basis_units<<<g2, 256, 0, st>>>(t->d_s1, cs, rm, nr, npsr, n_ph, P->n_r, nb, t->n_batches, dA);
        else
            k_basis<<<g2, 256, 0, st>>>(t->d_s1, cs, rm, nr, npsr, nb, t->n_batches, dA);
        count_launch();
        e = cudaGetLastError();
    }
    unsigned bad = 0;
    if (e == cudaSuccess && mem == LSM_MEM_HOST) {
        e = cudaMemcpyAsync(A, dA, (size_t)ncell * 8, cudaMemcpyDeviceToHost, st);
        // a phantom created without the host check: its verdict comes back too
        if (e == cudaSuccess && !ph->validated)
            e = cudaMemcpyAsync(&bad, ph->d_flags + 2, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFreeAsync(tmp, st);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_basis_matrix");
    if (bad) return set_arg_error("lsm_basis_matrix: the phantom's densities must be in [1e-4, 25] and materials in {0, 1}");
    return LSM_OK;
}

}  // namespace lsm
