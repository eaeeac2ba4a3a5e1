// common.cuh -- device-side building blocks shared by the kernels of liblsm.so.
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) counter RNG; the u32 ->
// (0,1] map; particle-queue and interaction-table layouts; launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lsm.h"

namespace lsm {

constexpr float kMe = 0.51099895f;       // electron rest energy, MeV
constexpr double kMeD = 0.51099895;
constexpr float kCutE = 0.2f;            // electron cutoff, MeV (Sec. 2.3)
constexpr float kCutG = 0.05f;           // photon cutoff, MeV (Sec. 2.3)
constexpr float kPi = 3.14159265358979f;
constexpr double kPiD = 3.14159265358979323846;
constexpr int kGrid = 1024;              // log-energy table points
constexpr double kLnEmin = -6.907755278982137;  // ln(1 keV in MeV)
constexpr double kLnEmax = 1.9459101090932196;  // ln(7 MeV)
// Inverse Klein-Nishina CDF table: v = (eta - 1) / (2k) as a function of
// (ln E, u), eta = E/E', k = E/mc^2; kKnE log-spaced energies 50 keV - 7 MeV,
// kKnU uniform u points on [0, 1].
constexpr int kKnE = 32, kKnU = 129;
constexpr double kKnLnE0 = -2.995732273553991;   // ln(0.05)
constexpr double kKnLnE1 = 1.9459101090932196;   // ln(7)

// ---------------------------------------------------------------- Philox ---
__device__ __forceinline__ uint4 philox4x32_10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                               uint32_t c2, uint32_t c3)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = c0 * 0xD2511F53u, hi0 = __umulhi(c0, 0xD2511F53u);
        const uint32_t lo1 = c2 * 0xCD9E8D57u, hi1 = __umulhi(c2, 0xCD9E8D57u);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ((x >> 8) + 1) * 2^-24: exact in FP32, never 0.
__device__ __forceinline__ float u01(uint32_t x)
{
    return __fmul_rn((float)(x >> 8) + 1.0f, 5.9604644775390625e-8f);
}

// A particle's random stream: counter (history lo, history hi, stream id, draw).
struct Stream {
    uint32_t k0, k1, glo, ghi, sid, ctr;
    uint32_t have;   // pre holds the block at counter ctr
    uint4 pre;
    __device__ __forceinline__ uint4 next()
    {
        const uint4 r = have ? pre : philox4x32_10(k0, k1, glo, ghi, sid, ctr);
        ++ctr;
        have = 0;
        return r;
    }
    // compute the block of the next draw ahead of time (same value next() returns)
    __device__ __forceinline__ void prefetch()
    {
        pre = philox4x32_10(k0, k1, glo, ghi, sid, ctr);
        have = 1;
    }
    // stream ids of the (up to four) particles created at the current draw
    // position: a hash of (stream id, draw counter, slot); ids 0 and 1 are
    // reserved for source sampling and primary transport
    __device__ __forceinline__ uint32_t child_id(uint32_t slot) const
    {
        uint32_t h = sid ^ fmix32(ctr ^ (0x9E3779B9u * (slot + 1u)));
        h = fmix32(h);
        return h < 2u ? h + 2u : h;
    }
    // MurmurHash3's 32-bit finaliser (Appleby)
    __device__ __forceinline__ static uint32_t fmix32(uint32_t h)
    {
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        h *= 0xC2B2AE35u;
        h ^= h >> 16;
        return h;
    }
};

// --------------------------------------------------------- particle queue ---
// Queue of particles waiting for transport, phantom-local coordinates
// (x - x0, y - y0, z - z0): three 16-byte words per particle, (x, y, z, E),
// (u, v, w, stream id bits), (history lo, history hi, PSR | beam << 16 |
// slot << 20, unused), so that a particle moves as one 48-byte record.
struct Queue {
    float4 *rec;
    uint32_t cap;
};

// Counters of one sample/transport iteration (device memory, zeroed per iteration).

// Each counter has a 128-byte line of its own: the photon pass's refill
// cursor and its pushes onto the electron queue are atomics from every
// warp, and on one shared line (with the pushes of the annihilation-photon
// queue of an earlier design) they queued
// behind one another in L2 (photon pass 0.49 -> 0.45 ms apart, with 64-slot
// output reservations).
struct alignas(128) CounterLine {
    uint32_t v;
    uint32_t unused[31];
    __host__ __device__ operator uint32_t &() { return v; }
    __host__ __device__ uint32_t *operator&() { return &v; }
};
struct IterCounters {
    CounterLine n[3];      // queue fill: 0 primary photons, 1 (unused), 2 electrons
    CounterLine head[3];   // refill cursors of the persistent transport kernels
    uint32_t overflow;     // electrons deposited in place because the queue was full
    uint32_t pad;          // table-staging timeout flag
    uint32_t src_e;        // electron-queue slots the source (sampler or a particle list) filled
    uint32_t dead;         // electron-queue slots photon warps reserved and left empty
};

// Run-long statistics and the FP64 energy ledger.
struct RunStats {
    double ledger[4];     // source, rejected, escaped, deposited (MeV)
    // histories, accepted photons, accepted electrons, rejected, missed,
    // Woodcock flights, real photon interactions, electron steps, step-cap
    // hits, queue overflows, electrons queued by photon transport
    unsigned long long c[11];
};

// ---------------------------------------------------- interaction tables ---
// Per material class: float4 (mu_compton, mu_photo, mu_pair [cm^2/g], S_col [MeV cm^2/g])
// at ln E_i = kLnEmin + i * dlnE; majorant [1/cm] per phantom.
struct Tables {
    const float4 *xs;    // [2][kGrid]
    const float *mumax;  // [kGrid]
    float inv_dlnE;
};

// ------------------------------------------------------------- warp utils ---
__device__ __forceinline__ unsigned lane_id()
{
    unsigned l;
    asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lsm

// ---------------------------------------------------------------- host side --
namespace lsm {
// Event timers around kernel groups (see lsm_timing_enable). timer_begin
// returns a token that timer_end closes; both are no-ops while disabled.
// a new process-wide unique id (plans and phantoms)
uint64_t next_uid();
int timer_begin(int which, cudaStream_t st);
void timer_end(int token, cudaStream_t st);
// timers recorded during a graph capture: detached after it, resolved per replay
size_t timer_mark();
void *timer_detach(size_t from);
void timer_replayed(void *set);
void timer_free(void *set);
void count_launch();
void add_launches(int64_t n);     // kernels launched by a replayed graph
bool timing_enabled();
lsm_status set_cuda_error(cudaError_t e, const char *where);
lsm_status set_arg_error(const char *msg);
lsm_status set_io_error(const char *what, const char *path, int err);
// Device memory from the device's stream-ordered pool (freed memory stays in
// the pool for the next allocation instead of going back to the driver):
// dev_malloc orders the allocation on `st`; dev_free returns it in the order
// of the legacy default stream (work on other streams must be complete).
cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p);
int sm_count();
}  // namespace lsm

#define LSM_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return lsm::set_cuda_error(_e, #call);    \
    } while (0)

#define LSM_LAUNCHED(where)                                              \
    do {                                                                 \
        lsm::count_launch();                                             \
        cudaError_t _e = cudaGetLastError();                             \
        if (_e != cudaSuccess) return lsm::set_cuda_error(_e, where);    \
    } while (0)
