// denoise.cu -- the dose denoiser: a BF16 3D U-Net on the tcgen05 tensor cores.
//
// A 3x3x3 convolution is an implicit GEMM D[m][o] = sum_k A[m][k] B[k][o]:
// m runs over 128 consecutive voxels of the padded volume (one M tile), o over
// output channels, k over (tap, input channel). Every activation volume keeps
// a one-voxel zero halo, so each tap is a pure shift of the padded linear voxel
// index by (dz-1) P + (dy-1) (w+2) + (dx-1), P = (h+2)(w+2). One pipeline stage
// covers one input-channel chunk (KC channels) and one dz: TMA loads three
// slabs of 130 voxels x KC channels (dy = 0, 1, 2, one voxel of x halo on
// either side), and the nine (dy, dx) taps of the stage are shared-memory
// descriptors that start dx rows into those slabs. The stage's weights arrive with one bulk copy,
// already packed into the operand layout on the host. Accumulators are FP32 in
// tensor memory, two per CTA so that the epilogue of one tile overlaps the MMAs
// of the next; the epilogue adds the bias, applies ReLU, writes BF16 and zeroes
// the halo voxels of the tile.
//
// Operand layouts in shared memory, both K-major: A (activations) in rows of
// 2 KC bytes with the 32/64/128-byte swizzle that TMA writes (SBO = 8 rows; a
// K = 16 step advances the start by 32 bytes; the swizzle phase follows the
// address, so a start shifted by whole rows reads the shifted rows); B
// (weights) without swizzle, core matrices of 8 rows x 16 bytes, SBO = 128
// bytes between 8-row groups, LBO between the two 8-element K halves.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "unet.cuh"

namespace lsm {
namespace dn {

constexpr int kTileM = 128;
constexpr int kSlabVox = kTileM + 2;            // one voxel of x halo either side
constexpr int kThreads = 192;                   // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
// drain bound after a give-up: copies and MMAs in flight finish in microseconds
constexpr unsigned long long kDrainNs = 100000000ull;

// A slab row is one voxel's KC input channels (2 KC bytes), stored with the
// matching TMA / UMMA swizzle (32, 64 or 128 bytes); slabs start on 1024-byte
// boundaries so that the swizzle phase of a row is that of its address.
template <int COUT, int KC>
struct Cfg {
    // fused (conv_fused): one MMA per (dz, dy, K step) covers the three dx
    // taps as N = 3 cout; each 128-row A tile is four 32-voxel boxes that
    // overlap by two voxels, so that every epilogue warp sums its outputs'
    // three dx contributions from its own TMEM lanes (30 outputs per warp)
    static constexpr bool kFused = conv_fused(COUT, KC);
    static constexpr int kRow = KC * 2;
    static constexpr int kSlabRows = kFused ? 128 : kSlabVox;
    static constexpr int kPitch = (kSlabRows * kRow + 1023) / 1024 * 1024;
    static constexpr int kA = 3 * kPitch;
    static constexpr int kB = 9 * COUT * KC * 2;
    static constexpr int kStage = (kA + kB + 1023) / 1024 * 1024;
    static constexpr int kBudget = kStage <= 50 * 1024 ? 100 * 1024 : 200 * 1024;
    static constexpr int kFit = kBudget / kStage;
    static constexpr int kStages = kFit < 2 ? 2 : (kFit > 8 ? 8 : kFit);
    static constexpr int kTx = 3 * kSlabRows * kRow + kB;
    static constexpr uint32_t kSwz = KC == 16 ? 6u : (KC == 32 ? 4u : 2u);   // 32B, 64B, 128B swizzle
    static constexpr int kN = kFused ? 3 * COUT : COUT;
    static constexpr int kAccCols = kFused ? (3 * COUT + 31) / 32 * 32 : (COUT < 32 ? 32 : COUT);
    static constexpr int kTmemCols = 2 * kAccCols <= 64 ? 64 : (2 * kAccCols <= 128 ? 128 : (2 * kAccCols <= 256 ? 256 : 512));
    static constexpr int kTileOut = kFused ? 120 : kTileM;   // output voxels per tile
    static constexpr int kSmem = kStages * kStage + 1024;
    static_assert(KC == 16 || KC == 32 || KC == 64, "channel chunk");
    static_assert(2 * kAccCols <= kTmemCols && kTmemCols <= 512, "tensor memory columns");
    static_assert(kN % 16 == 0 && kN <= 256, "MMA N");
};

struct ConvArgs {
    const __nv_bfloat16 *wimg;
    const float *bias;
    __nv_bfloat16 *out;
    long long lp;             // padded voxels per volume
    long long l0;             // padded index of the first interior voxel
    int out_ct, out_co, in_co;
    int n_kc;
    int w2, p;                // w + 2, (h + 2)(w + 2)
    int d, h, w;
    int tiles_per_vol, n_tiles;
    int relu;
    unsigned *err;
    unsigned long long wait_ns;   // bound of each pipeline wait (lsm_set_wait_limits)
};

// ------------------------------------------------------------ PTX helpers ---
__device__ __forceinline__ uint32_t s2u(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mb_init(uint64_t *b, unsigned n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s2u(b)), "r"(n) : "memory");
}

__device__ __forceinline__ void mb_expect(uint64_t *b, unsigned tx)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s2u(b)), "r"(tx) : "memory");
}

__device__ __forceinline__ void mb_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s2u(b)) : "memory");
}

__device__ __forceinline__ bool mb_test(uint64_t *b, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(s2u(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete. Bounded: after wait_ns,
// or when another role has given up, returns false; a timeout sets `code` in
// *err and the CTA's abort flag.
__device__ bool mb_wait(uint64_t *b, unsigned parity, volatile int *abort_flag, unsigned *err, unsigned code,
                        unsigned long long wait_ns)
{
    if (mb_test(b, parity)) return true;
    const unsigned long long t0 = gtime();
    for (;;) {
        if (mb_test(b, parity)) return true;
        if (*abort_flag) return false;
        if (gtime() - t0 > wait_ns) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}

// After the pipeline stops (normally or after a give-up): wait, bounded by
// kDrainNs and ignoring the abort flag, for a phase the CTA's own copies or
// tensor-core operations will complete, so that none is in flight when the
// CTA releases its tensor memory and exits. A drain that runs out sets 16.
__device__ void mb_drain(uint64_t *b, unsigned parity, unsigned *err)
{
    if (mb_test(b, parity)) return;
    const unsigned long long t0 = gtime();
    while (!mb_test(b, parity)) {
        if (gtime() - t0 > kDrainNs) {
            atomicOr(err, 16u);
            return;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(s2u(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(s2u(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(s2u(bar))
                 : "memory");
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (16-byte units), descriptor version 1, layout (0 none, 6 32B, 4 64B, 2 128B swizzle)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout = 0)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s2u(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------ conv kernel ---
template <int COUT, int KC>
__global__ void __launch_bounds__(kThreads, 1) k_conv3d(const __grid_constant__ CUtensorMap tin, const ConvArgs a)
{
    using C = Cfg<COUT, KC>;
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[C::kStages], empty[C::kStages], accf[2], acce[2], mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const uint32_t sbase = (s2u(dsm) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mb_init(&accf[i], 1);
            mb_init(&acce[i], 4);
        }
        mb_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s2u(&tmem_slot)),
                     "r"(C::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_slot;
    const int ksteps = a.n_kc * 3;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tin) : "memory");
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < a.n_tiles && ok; t += gridDim.x) {
                const int vol = t / a.tiles_per_vol;
                const long long lt = a.l0 + (long long)(t - vol * a.tiles_per_vol) * C::kTileOut;
                for (int k = 0; k < ksteps; ++k, ++it) {
                    const int s = it % C::kStages;
                    if (it >= C::kStages &&
                        !mb_wait(&empty[s], (unsigned)((it / C::kStages) - 1) & 1u, &abort_flag, a.err, 1u, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const int kc = k / 3, dz = k - 3 * kc;
                    const uint32_t sa = sbase + (uint32_t)(s * C::kStage), sb = sa + C::kA;
                    mb_expect(&full[s], C::kTx);
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
                        const int c1 = (int)(lt - 1 + (long long)(dz - 1) * a.p + (long long)(dy - 1) * a.w2);
                        if constexpr (C::kFused) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)   // rows 32 q .. 32 q + 31: voxels c1 + 30 q ..
                                tma_load_3d(sa + (uint32_t)(dy * C::kPitch + q * 32 * C::kRow), &tin,
                                            a.in_co + kc * KC, c1 + 30 * q, vol, &full[s]);
                        } else {
                            tma_load_3d(sa + (uint32_t)(dy * C::kPitch), &tin, a.in_co + kc * KC, c1, vol, &full[s]);
                        }
                    }
                    bulk_load(sb, a.wimg + (size_t)(kc * 3 + dz) * 9 * COUT * KC, C::kB, &full[s]);
                }
            }
            // loads issued (it of them) land before the CTA moves on: the
            // newest phase of each stage's full barrier (already complete
            // unless the pipeline stopped early)
            for (int j = it > C::kStages ? it - C::kStages : 0; j < it; ++j)
                mb_drain(&full[j % C::kStages], (unsigned)(j / C::kStages) & 1u, a.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = (1u << 4)      // D: FP32
                                       | (1u << 7)    // A: BF16
                                       | (1u << 10)   // B: BF16
                                       | ((uint32_t)(C::kN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
            int it = 0, li = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < a.n_tiles && ok; t += gridDim.x, ++li) {
                const int acc = li & 1;
                if (li >= 2 && !mb_wait(&acce[acc], (unsigned)((li >> 1) - 1) & 1u, &abort_flag, a.err, 2u, a.wait_ns))
                    break;
                tc_after();
                const uint32_t d = tmem + (uint32_t)(acc * C::kAccCols);
                for (int k = 0; k < ksteps; ++k, ++it) {
                    const int s = it % C::kStages;
                    if (!mb_wait(&full[s], (unsigned)(it / C::kStages) & 1u, &abort_flag, a.err, 4u, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_after();
                    const uint32_t sa = sbase + (uint32_t)(s * C::kStage), sb = sa + C::kA;
                    if constexpr (C::kFused) {
                        // the dx taps are N groups of one operand: A starts at row 0
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int j = 0; j < KC / 16; ++j) {
                                const uint64_t ad =
                                    sdesc(sa + (uint32_t)(dy * C::kPitch + j * 32), 16, 8 * C::kRow, C::kSwz);
                                const uint64_t bd = sdesc(
                                    sb + (uint32_t)(dy * (3 * COUT * KC * 2) + j * 2 * (3 * COUT * 16)), 3 * COUT * 16,
                                    128);
                                mma_bf16(d, ad, bd, idesc, (k | dy | j) != 0);
                            }
                    } else {
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                                for (int j = 0; j < KC / 16; ++j) {
                                    const uint64_t ad = sdesc(sa + (uint32_t)(dy * C::kPitch + dx * C::kRow + j * 32),
                                                              16, 8 * C::kRow, C::kSwz);
                                    const uint64_t bd = sdesc(
                                        sb + (uint32_t)((dy * 3 + dx) * (COUT * KC * 2) + j * 2 * (COUT * 16)),
                                        COUT * 16, 128);
                                    mma_bf16(d, ad, bd, idesc, (k | dy | dx | j) != 0);
                                }
                    }
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&accf[acc]);
            }
            // every MMA this thread issued has completed before tensor memory is released
            mma_commit(&mma_done);
            mb_drain(&mma_done, 0u, a.err);
        }
    } else {   // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int q = warp & 3;
        int li = 0;
        for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x, ++li) {
            const int acc = li & 1;
            const bool ok = mb_wait(&accf[acc], (unsigned)(li >> 1) & 1u, &abort_flag, a.err, 8u, a.wait_ns);
            if (!__all_sync(0xFFFFFFFFu, ok)) break;
            tc_after();
            const int vol = t / a.tiles_per_vol;
            const long long lt = a.l0 + (long long)(t - vol * a.tiles_per_vol) * C::kTileOut;
            if constexpr (C::kFused) {
                // lane j of quarter q holds row 32 q + j = input voxel lt - 1 + 30 q + j;
                // output lt + 30 q + j (j < 30) = P0[j] + P1[j + 1] + P2[j + 2]
                const long long L = lt + 30 * q + lane;
                const long long zz = L / a.p;
                const int rem = (int)(L - zz * a.p);
                const int yy = rem / a.w2, xx = rem - yy * a.w2;
                const bool inside = zz >= 1 && zz <= a.d && yy >= 1 && yy <= a.h && xx >= 1 && xx <= a.w;
                const bool write = lane < 30 && L < a.lp;
                __nv_bfloat16 *o = a.out + ((size_t)vol * (size_t)a.lp + (size_t)(write ? L : 0)) * a.out_ct + a.out_co;
                const uint32_t row = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * C::kAccCols);
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    uint32_t r0[16], r1[16], r2[16];
                    tmem_ld16(row + (uint32_t)c0, r0);
                    tmem_ld16(row + (uint32_t)(COUT + c0), r1);
                    tmem_ld16(row + (uint32_t)(2 * COUT + c0), r2);
                    uint32_t pk[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float v[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int c = 2 * i + h;
                            const float p1 = __shfl_down_sync(0xFFFFFFFFu, __uint_as_float(r1[c]), 1);
                            const float p2 = __shfl_down_sync(0xFFFFFFFFu, __uint_as_float(r2[c]), 2);
                            float x = __uint_as_float(r0[c]) + p1 + p2 + __ldg(a.bias + c0 + c);
                            if (a.relu) x = fmaxf(x, 0.0f);
                            v[h] = inside ? x : 0.0f;
                        }
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[0], v[1]);
                        pk[i] = *reinterpret_cast<const uint32_t *>(&h2);
                    }
                    if (write) {
                        uint4 *dst = reinterpret_cast<uint4 *>(o + c0);
                        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    }
                }
                tc_before();
                __syncwarp();
                if (lane == 0) mb_arrive(&acce[acc]);
                continue;
            }
            const long long L = lt + 32 * q + lane;
            const long long zz = L / a.p;
            const int rem = (int)(L - zz * a.p);
            const int yy = rem / a.w2, xx = rem - yy * a.w2;
            const bool inside = zz >= 1 && zz <= a.d && yy >= 1 && yy <= a.h && xx >= 1 && xx <= a.w;
            const bool write = L < a.lp;
            __nv_bfloat16 *o = a.out + ((size_t)vol * (size_t)a.lp + (size_t)(write ? L : 0)) * a.out_ct + a.out_co;
#pragma unroll
            for (int c0 = 0; c0 < COUT; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * C::kAccCols + c0), r);
                uint32_t pk[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float v0 = __uint_as_float(r[2 * i]) + __ldg(a.bias + c0 + 2 * i);
                    float v1 = __uint_as_float(r[2 * i + 1]) + __ldg(a.bias + c0 + 2 * i + 1);
                    if (a.relu) {
                        v0 = fmaxf(v0, 0.0f);
                        v1 = fmaxf(v1, 0.0f);
                    }
                    if (!inside) v0 = v1 = 0.0f;
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                    pk[i] = *reinterpret_cast<const uint32_t *>(&h2);
                }
                if (write) {
                    uint4 *dst = reinterpret_cast<uint4 *>(o + c0);
                    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
            tc_before();
            __syncwarp();
            if (lane == 0) mb_arrive(&acce[acc]);
        }
    }
    __syncwarp();
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------- memory-bound kernels ---
__device__ __forceinline__ uint4 max8(uint4 a, uint4 b)
{
    uint4 r;
    const __nv_bfloat162 *x = reinterpret_cast<const __nv_bfloat162 *>(&a);
    const __nv_bfloat162 *y = reinterpret_cast<const __nv_bfloat162 *>(&b);
    __nv_bfloat162 *z = reinterpret_cast<__nv_bfloat162 *>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) z[i] = __hmax2(x[i], y[i]);
    return r;
}

// 2x2x2 max pooling; one thread per (output voxel, 8-channel group)
__global__ void k_pool2(const __nv_bfloat16 *__restrict__ in, int in_ct, int in_co, __nv_bfloat16 *__restrict__ out,
                        int out_ct, int out_co, int groups, int n, VolIdx vo, VolIdx vi)
{
    const long long total = (long long)n * vo.d * vo.h * vo.w * groups;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % groups);
        long long v = i / groups;
        const int x = (int)(v % vo.w); v /= vo.w;
        const int y = (int)(v % vo.h); v /= vo.h;
        const int z = (int)(v % vo.d);
        const int b = (int)(v / vo.d);
        uint4 m = make_uint4(0xFF80FF80u, 0xFF80FF80u, 0xFF80FF80u, 0xFF80FF80u);   // -inf
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const long long src = vi.at(b, 2 * z + (c >> 2), 2 * y + ((c >> 1) & 1), 2 * x + (c & 1));
            m = max8(m, *reinterpret_cast<const uint4 *>(in + src * in_ct + in_co + 8 * g));
        }
        *reinterpret_cast<uint4 *>(out + vo.at(b, z, y, x) * out_ct + out_co + 8 * g) = m;
    }
}

// nearest 2x upsampling; one thread per (output voxel, 8-channel group)
__global__ void k_up2(const __nv_bfloat16 *__restrict__ in, int in_ct, int in_co, __nv_bfloat16 *__restrict__ out,
                      int out_ct, int out_co, int groups, int n, VolIdx vo, VolIdx vi)
{
    const long long total = (long long)n * vo.d * vo.h * vo.w * groups;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % groups);
        long long v = i / groups;
        const int x = (int)(v % vo.w); v /= vo.w;
        const int y = (int)(v % vo.h); v /= vo.h;
        const int z = (int)(v % vo.d);
        const int b = (int)(v / vo.d);
        *reinterpret_cast<uint4 *>(out + vo.at(b, z, y, x) * out_ct + out_co + 8 * g) =
            *reinterpret_cast<const uint4 *>(in + vi.at(b, z >> 1, y >> 1, x >> 1) * in_ct + in_co + 8 * g);
    }
}

// per-volume maximum of a non-negative FP32 dose (float bits compare as ints)
__global__ void k_dmax(const float *__restrict__ dose, long long per_vol, int n, unsigned *dmax_bits)
{
    for (int b = blockIdx.y; b < n; b += gridDim.y) {
        unsigned m = 0;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per_vol;
             i += (long long)gridDim.x * blockDim.x)
            m = max(m, __float_as_uint(fmaxf(dose[(long long)b * per_vol + i], 0.0f)));
        for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax(dmax_bits + b, m);
    }
}

// input volume: channel 0 dose / Dmax, channel 1 density, channels 2-15 zero
__global__ void k_pack_input(const float *__restrict__ dose, const float *__restrict__ rho,
                             const unsigned *__restrict__ dmax_bits, __nv_bfloat16 *__restrict__ x, int n, VolIdx v)
{
    const long long per = (long long)v.d * v.h * v.w, total = per * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / per);
        long long r = i - (long long)b * per;
        const int xx = (int)(r % v.w); r /= v.w;
        const int yy = (int)(r % v.h);
        const int zz = (int)(r / v.h);
        const double dm = (double)__uint_as_float(dmax_bits[b]);
        const double sc = dm > 0.0 ? 1.0 / dm : 0.0;
        const float d0 = __double2float_rn((double)dose[i] * sc);
        const __nv_bfloat162 h = __halves2bfloat162(__float2bfloat16_rn(d0), __float2bfloat16_rn(rho[i]));
        uint4 *dst = reinterpret_cast<uint4 *>(x + v.at(b, zz, yy, xx) * 16);
        dst[0] = make_uint4(*reinterpret_cast<const uint32_t *>(&h), 0u, 0u, 0u);
        dst[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// out = dose + Dmax * (sum_c hw[c] d0[c] + hb)
__global__ void k_head(const __nv_bfloat16 *__restrict__ d0, int ct, const float *__restrict__ hw,
                       const float *__restrict__ dose, const unsigned *__restrict__ dmax_bits, float *__restrict__ out,
                       int n, VolIdx v)
{
    const long long per = (long long)v.d * v.h * v.w, total = per * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / per);
        long long r = i - (long long)b * per;
        const int xx = (int)(r % v.w); r /= v.w;
        const int yy = (int)(r % v.h);
        const int zz = (int)(r / v.h);
        const uint4 *src = reinterpret_cast<const uint4 *>(d0 + v.at(b, zz, yy, xx) * ct);
        float acc = hw[16];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint4 u = src[k];
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 f = __bfloat1622float2(h[j]);
                acc += hw[8 * k + 2 * j] * f.x + hw[8 * k + 2 * j + 1] * f.y;
            }
        }
        out[i] = dose[i] + __uint_as_float(dmax_bits[b]) * acc;
    }
}

// interior voxels of channels [co, co + c) -> dense [n][d][h][w][c]
__global__ void k_extract(const __nv_bfloat16 *__restrict__ in, int ct, int co, int c, __nv_bfloat16 *__restrict__ dst,
                          int n, VolIdx v)
{
    const long long per = (long long)v.d * v.h * v.w, total = per * n * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int b = (int)(r / per);
        r -= (long long)b * per;
        const int xx = (int)(r % v.w); r /= v.w;
        const int yy = (int)(r % v.h);
        const int zz = (int)(r / v.h);
        dst[i] = in[v.at(b, zz, yy, xx) * ct + co + ch];
    }
}

// ------------------------------------------------------------------- host ---
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    }
    return fn;
}

// bound of each pipeline wait of the convolution kernels (lsm_set_wait_limits)
unsigned long long g_conv_wait_ns = 2000000000ull;

unsigned *g_err_word = nullptr;
unsigned *err_word()
{
    if (!g_err_word) {
        if (cudaMalloc(&g_err_word, 16) != cudaSuccess) return nullptr;
        cudaMemset(g_err_word, 0, 16);
    }
    return g_err_word;
}

lsm_status check_vol(const lsm_vol *v, const char *what)
{
    char msg[160];
    if (!v || !v->data) {
        snprintf(msg, sizeof msg, "%s: NULL volume", what);
        return set_arg_error(msg);
    }
    if (v->n < 1 || v->d < 1 || v->h < 1 || v->w < 1 || v->c_total < 8 || v->c_total % 8 || v->c_offset < 0 ||
        v->c_offset % 8 || v->c < 8 || v->c % 8 || v->c_offset + v->c > v->c_total ||
        ((uintptr_t)v->data & 15)) {
        snprintf(msg, sizeof msg, "%s: bad volume (sizes >= 1; channels multiples of 8 within c_total; 16-byte base)",
                 what);
        return set_arg_error(msg);
    }
    return LSM_OK;
}

template <int COUT, int KC>
lsm_status launch_conv(const CUtensorMap &map, const ConvArgs &a, int ctas_per_sm, cudaStream_t st)
{
    using C = Cfg<COUT, KC>;
    static int occ = 0;
    if (!occ) {
        LSM_CUDA(cudaFuncSetAttribute(k_conv3d<COUT, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
        // The occupancy query answers 1 for any kernel holding tcgen05
        // instructions, whatever it uses; count the resident CTAs from the
        // shared memory, the 512 tensor-memory columns, registers and warps.
        cudaFuncAttributes fa;
        LSM_CUDA(cudaFuncGetAttributes(&fa, k_conv3d<COUT, KC>));
        int dev = 0, smem_sm = 0, rsv = 0;
        LSM_CUDA(cudaGetDevice(&dev));
        LSM_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        LSM_CUDA(cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        const int by_smem = smem_sm / (C::kSmem + (int)fa.sharedSizeBytes + rsv);
        const int by_tmem = 512 / C::kTmemCols;
        const int by_regs = 65536 / (((fa.numRegs + 7) / 8 * 8) * kThreads);
        const int by_warps = 64 / (kThreads / 32);
        occ = std::max(1, std::min(std::min(by_smem, by_tmem), std::min(by_regs, by_warps)));
    }
    const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
    const int grid = std::max(1, std::min(a.n_tiles, per_sm * sm_count()));
    k_conv3d<COUT, KC><<<grid, kThreads, C::kSmem, st>>>(map, a);
    count_launch();
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

// input channels per stage: weights of a stage (9 taps x cout x kc) stay <= 36 KB
int kc_for(int cin, int cout)
{
    const int kmax = cout >= 128 ? 16 : (cout == 64 ? 32 : 64);
    return std::min(cin, kmax);
}

lsm_status conv_forward(const lsm_conv3d *cv, const lsm_vol *in, const lsm_vol *out, int ctas_per_sm,
                        cudaStream_t st)
{
    if (!cv) return set_arg_error("lsm_conv3d_forward: NULL layer");
    lsm_status rc = check_vol(in, "lsm_conv3d_forward input");
    if (rc) return rc;
    if ((rc = check_vol(out, "lsm_conv3d_forward output"))) return rc;
    if (in->n != out->n || in->d != out->d || in->h != out->h || in->w != out->w)
        return set_arg_error("lsm_conv3d_forward: input and output sizes differ");
    if (in->c != cv->cin || out->c != cv->cout) return set_arg_error("lsm_conv3d_forward: channel counts");
    const VolIdx v = vidx(in->d, in->h, in->w);
    if (v.lp >= (1ll << 31) - 4096) return set_arg_error("lsm_conv3d_forward: volume too large");
    EncodeTiled enc = encode_fn();
    if (!enc) return set_arg_error("lsm_conv3d_forward: cuTensorMapEncodeTiled unavailable");
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)in->c_total, (cuuint64_t)v.lp, (cuuint64_t)in->n};
    const cuuint64_t strides[2] = {(cuuint64_t)in->c_total * 2, (cuuint64_t)v.lp * in->c_total * 2};
    const bool fused = conv_fused(cv->cout, cv->kc);
    const cuuint32_t box[3] = {(cuuint32_t)cv->kc, (cuuint32_t)(fused ? 32 : kSlabVox), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapSwizzle swz = cv->kc == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                   : cv->kc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, in->data, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        char msg[96];
        snprintf(msg, sizeof msg, "lsm_conv3d_forward: tensor map encoding failed (%d)", (int)cr);
        return set_arg_error(msg);
    }
    unsigned *err = err_word();
    if (!err) return set_cuda_error(cudaErrorMemoryAllocation, "lsm_conv3d_forward: error word");
    ConvArgs a;
    a.wimg = cv->wimg;
    a.bias = cv->bias;
    a.out = (__nv_bfloat16 *)out->data;
    a.lp = v.lp;
    // tiled span: from the x halo before the first interior voxel to the one
    // after the last, so that interior rows are written whole
    a.l0 = (long long)v.p + v.w2;
    const long long llast = (long long)in->d * v.p + (long long)in->h * v.w2 + in->w + 1;
    const int tile_out = fused ? 120 : kTileM;      // Cfg<>::kTileOut
    a.tiles_per_vol = (int)((llast - a.l0 + tile_out) / tile_out);
    a.n_tiles = a.tiles_per_vol * in->n;
    a.out_ct = out->c_total;
    a.out_co = out->c_offset;
    a.in_co = in->c_offset;
    a.n_kc = cv->cin / cv->kc;
    a.w2 = v.w2;
    a.p = v.p;
    a.d = in->d; a.h = in->h; a.w = in->w;
    a.relu = cv->relu;
    a.err = err;
    a.wait_ns = g_conv_wait_ns;
    const int tk = timer_begin(8, st);
    lsm_status r = LSM_ERR_ARG;
    switch (cv->cout * 1000 + cv->kc) {
    case 16016: r = launch_conv<16, 16>(map, a, ctas_per_sm, st); break;
    case 16032: r = launch_conv<16, 32>(map, a, ctas_per_sm, st); break;
    case 16064: r = launch_conv<16, 64>(map, a, ctas_per_sm, st); break;
    case 32016: r = launch_conv<32, 16>(map, a, ctas_per_sm, st); break;
    case 32032: r = launch_conv<32, 32>(map, a, ctas_per_sm, st); break;
    case 32064: r = launch_conv<32, 64>(map, a, ctas_per_sm, st); break;
    case 64016: r = launch_conv<64, 16>(map, a, ctas_per_sm, st); break;
    case 64032: r = launch_conv<64, 32>(map, a, ctas_per_sm, st); break;
    case 128016: r = launch_conv<128, 16>(map, a, ctas_per_sm, st); break;
    default: set_arg_error("lsm_conv3d_forward: unsupported channel configuration");
    }
    timer_end(tk, st);
    return r;
}

lsm_status conv_create(int cin, int cout, int relu, const float *w, const float *b, lsm_conv3d **out,
                       cudaStream_t st)
{
    if (!out || !w) return set_arg_error("lsm_conv3d_create: NULL argument");
    auto okc = [](int c) { return c == 16 || c == 32 || c == 64 || c == 128; };
    if (!okc(cin) || !okc(cout)) return set_arg_error("lsm_conv3d_create: channels must be 16, 32, 64 or 128");
    const int kc = kc_for(cin, cout);
    const size_t nw = (size_t)27 * cin * cout;
    std::vector<__nv_bfloat16> img(nw);
    for (int c = 0; c < cin / kc; ++c)
        for (int dz = 0; dz < 3; ++dz)
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap % 3;
                for (int n = 0; n < cout; ++n)
                    for (int k = 0; k < kc; ++k)
                        img[wimg_offset(cout, kc, c, dz, dy, dx, n, k)] =
                            __float2bfloat16_rn(w[((((size_t)n * 3 + dz) * 3 + dy) * 3 + dx) * cin + c * kc + k]);
            }
    std::vector<float> bias(cout, 0.0f);
    for (int n = 0; n < cout && b; ++n) bias[n] = __bfloat162float(__float2bfloat16_rn(b[n]));
    lsm_conv3d *cv = nullptr;
    lsm_status rc = conv_alloc(cin, cout, relu, &cv);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(cv->wimg, img.data(), nw * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cv->bias, bias.data(), (size_t)cout * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        conv_destroy(cv);
        return set_cuda_error(e, "lsm_conv3d_create");
    }
    *out = cv;
    return LSM_OK;
}

// a layer's device buffers (weights image and bias), contents unset
lsm_status conv_alloc(int cin, int cout, int relu, lsm_conv3d **out)
{
    auto okc = [](int c) { return c == 16 || c == 32 || c == 64 || c == 128; };
    if (!okc(cin) || !okc(cout)) return set_arg_error("lsm_conv3d: channels must be 16, 32, 64 or 128");
    lsm_conv3d *cv = (lsm_conv3d *)calloc(1, sizeof(lsm_conv3d));
    if (!cv) return set_arg_error("lsm_conv3d: out of host memory");
    cv->cin = cin; cv->cout = cout; cv->relu = relu ? 1 : 0; cv->kc = kc_for(cin, cout);
    cudaError_t e = cudaMalloc(&cv->wimg, (size_t)27 * cin * cout * 2);
    if (e == cudaSuccess) e = cudaMalloc(&cv->bias, (size_t)cout * 4);
    if (e == cudaSuccess) e = cudaMemset(cv->bias, 0, (size_t)cout * 4);
    if (e != cudaSuccess) {
        conv_destroy(cv);
        return set_cuda_error(e, "lsm_conv3d: device memory");
    }
    *out = cv;
    return LSM_OK;
}

void conv_destroy(lsm_conv3d *cv)
{
    if (!cv) return;
    cudaFree(cv->wimg);
    cudaFree(cv->bias);
    free(cv);
}

int grid_1d(long long work)
{
    return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, 16ll * sm_count()));
}

lsm_status pool_or_up(const lsm_vol *in, const lsm_vol *out, bool up, cudaStream_t st)
{
    const char *name = up ? "lsm_upsample3d" : "lsm_pool3d";
    lsm_status rc = check_vol(in, name);
    if (rc) return rc;
    if ((rc = check_vol(out, name))) return rc;
    const bool sizes = up ? (out->d == 2 * in->d && out->h == 2 * in->h && out->w == 2 * in->w)
                          : (in->d == 2 * out->d && in->h == 2 * out->h && in->w == 2 * out->w);
    if (!sizes || in->n != out->n || in->c != out->c) {
        char msg[96];
        snprintf(msg, sizeof msg, "%s: sizes must halve/double and channel counts match", name);
        return set_arg_error(msg);
    }
    const VolIdx vi = vidx(in->d, in->h, in->w), vo = vidx(out->d, out->h, out->w);
    const int groups = in->c / 8;
    const long long work = (long long)out->n * out->d * out->h * out->w * groups;
    const int tk = timer_begin(9, st);
    if (up)
        k_up2<<<grid_1d(work), 256, 0, st>>>((const __nv_bfloat16 *)in->data, in->c_total, in->c_offset,
                                              (__nv_bfloat16 *)out->data, out->c_total, out->c_offset, groups, out->n,
                                              vo, vi);
    else
        k_pool2<<<grid_1d(work), 256, 0, st>>>((const __nv_bfloat16 *)in->data, in->c_total, in->c_offset,
                                                (__nv_bfloat16 *)out->data, out->c_total, out->c_offset, groups,
                                                out->n, vo, vi);
    count_launch();
    timer_end(tk, st);
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

// ------------------------------------------ weight gradient on tcgen05 ---
// dW[o][t][c] = sum over interior voxels v of gz[v][o] x[v + off_t][c], t =
// (dz, dy, dx). The contraction runs over voxels, so voxels are the MMA's K.
// The activations are voxel-major (channels contiguous), while the operands
// below are K-major, and a tap's offset off_t = (dz-1)P + (dy-1)(w+2) + dx-1
// is not a multiple of the 8 voxels (16 bytes) a TMA start or a matrix
// descriptor can move by. So a transposition pass first writes channel-major
// copies in a layout L8 whose row pitch W8 = roundup(w + 2, 8) and plane pitch
// P8 = (h + 2) W8 are multiples of 8: three copies of x, copy k holding the
// value at L8 index u + k - 1 (the dx shift), and one of gz. Tap t's operand
// then starts at u0 + (dz-1) P8 + (dy-1) W8, a multiple of 8 when u0 is.
//
// GEMM: M = 128 rows of (tap, input channel) pairs (128 / cin taps per row
// tile, 27 taps in ceil(27 cin / 128) tiles), N = cout, K = voxels in chunks
// of 64 (one 128-byte swizzled row per operand row). A CTA owns one row tile
// and a range of chunks of one volume: TMA loads (128 / cin boxes for A, one
// for B per stage), one thread issues the MMAs into one TMEM accumulator,
// four warps read it at the end and add it to dW with FP32 atomics.

struct L8 {
    int d, h, w, w8;
    long long p8, lq;         // plane pitch, voxels per volume copy
};

inline L8 l8_of(int d, int h, int w)
{
    L8 q;
    q.d = d; q.h = h; q.w = w;
    q.w8 = (w + 2 + 7) / 8 * 8;
    q.p8 = (long long)(h + 2) * q.w8;
    q.lq = (long long)(d + 2) * q.p8;
    return q;
}

// out[((b ncopy + k) c + ch) lq + u] = in at the L8 index u + shift_k (shift_k
// = k - 1 with three copies, 0 with one) if that voxel is interior, else 0.
// A CTA transposes 64 consecutive u of one (volume, copy) for all c channels
// through shared memory, reading 16-byte channel groups and writing 128-byte
// voxel rows.
__global__ void __launch_bounds__(256) k_chmajor(const __nv_bfloat16 *__restrict__ in, int ct, int co, int c, VolIdx v,
                                                 L8 q, int ncopy, __nv_bfloat16 *__restrict__ out)
{
    __shared__ __nv_bfloat16 tile[64 * (128 + 2)];
    const int pitch = c + 2;
    const long long u0 = (long long)blockIdx.x * 64;
    const int k = blockIdx.y % ncopy, b = blockIdx.y / ncopy;
    const int shift = ncopy == 3 ? k - 1 : 0;
    const int groups = c / 8;
    for (int i = threadIdx.x; i < 64 * groups; i += blockDim.x) {
        const int uu = i / groups, g = i - uu * groups;
        const long long u = u0 + uu + shift;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (u >= 0 && u < q.lq && u0 + uu < q.lq) {
            const long long z = u / q.p8, r = u - z * q.p8;
            const int y = (int)(r / q.w8), x = (int)(r - (long long)y * q.w8);
            if (z >= 1 && z <= q.d && y >= 1 && y <= q.h && x >= 1 && x <= q.w) {
                const long long src = (long long)b * v.lp + z * v.p + (long long)y * v.w2 + x;
                val = *reinterpret_cast<const uint4 *>(in + src * ct + co + g * 8);
            }
        }
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&val);
#pragma unroll
        for (int j = 0; j < 8; ++j) tile[uu * pitch + g * 8 + j] = e[j];
    }
    __syncthreads();
    __nv_bfloat16 *o = out + ((long long)blockIdx.y * c) * q.lq + u0;
    for (int i = threadIdx.x; i < 32 * c; i += blockDim.x) {
        const int ch = i / 32, pr = i - ch * 32;      // voxels 2 pr, 2 pr + 1 of channel ch
        if (u0 + 2 * pr + 1 < q.lq) {
            __nv_bfloat162 two;
            two.x = tile[(2 * pr) * pitch + ch];
            two.y = tile[(2 * pr + 1) * pitch + ch];
            *reinterpret_cast<__nv_bfloat162 *>(o + (long long)ch * q.lq + 2 * pr) = two;
        }
    }
}

template <int COUT, int CIN>
struct WgCfg {
    static constexpr int kTpt = 128 / CIN;                  // taps per row tile
    static constexpr int kMt = (27 + kTpt - 1) / kTpt;      // row tiles
    static constexpr int kA = 128 * 128;                    // 128 rows x 64 voxels, BF16
    static constexpr int kB = COUT * 128;
    static constexpr int kStage = kA + kB;                  // multiple of 1024
    static constexpr int kStages = kStage <= 20 * 1024 ? 5 : 4;
    static constexpr int kTx = kA + kB;
    static constexpr int kCols = COUT < 32 ? 32 : COUT;     // TMEM columns (power of 2)
    static constexpr int kSmem = kStages * kStage + 1024;
    static_assert(CIN == 16 || CIN == 32 || CIN == 64 || CIN == 128, "cin");
    static_assert(COUT % 16 == 0 && COUT <= 128, "cout");
};

struct WgArgs {
    float *dw;                // [cout][27][cin], accumulated
    L8 q;
    long long u_first;        // first chunk start (multiple of 64)
    int n_chunks;             // chunks of 64 voxels per volume
    int ksplit;               // CTAs per (volume, row tile)
    unsigned *err;
    unsigned long long wait_ns;
};

template <int COUT, int CIN>
__global__ void __launch_bounds__(kThreads, 1) k_wgrad_tc(const __grid_constant__ CUtensorMap mx,
                                                        const __grid_constant__ CUtensorMap mg, const WgArgs a)
{
    using C = WgCfg<COUT, CIN>;
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[C::kStages], empty[C::kStages], accf, mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const uint32_t sbase = (s2u(dsm) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ks = blockIdx.x % a.ksplit;
    const int mt = (blockIdx.x / a.ksplit) % C::kMt;
    const int vol = blockIdx.x / (a.ksplit * C::kMt);
    const int per = (a.n_chunks + a.ksplit - 1) / a.ksplit;
    const int c0 = ks * per, c1 = min(a.n_chunks, c0 + per);
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        mb_init(&accf, 1);
        mb_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s2u(&tmem_slot)),
                     "r"(C::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_slot;
    const int nk = c1 > c0 ? c1 - c0 : 0;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&mx) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&mg) : "memory");
            int it = 0;
            for (; it < nk; ++it) {
                const int s = it % C::kStages;
                if (it >= C::kStages &&
                    !mb_wait(&empty[s], (unsigned)((it / C::kStages) - 1) & 1u, &abort_flag, a.err, 1u, a.wait_ns))
                    break;
                const uint32_t sa = sbase + (uint32_t)(s * C::kStage), sb = sa + C::kA;
                const long long u0 = a.u_first + (long long)(c0 + it) * 64;
                mb_expect(&full[s], C::kTx);
#pragma unroll
                for (int k = 0; k < C::kTpt; ++k) {
                    // rows of taps past the 27th (last row tile) load tap 26's
                    // box again; the epilogue drops them
                    const int t = min(mt * C::kTpt + k, 26);
                    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                    const int ux = (int)(u0 + (long long)(dz - 1) * a.q.p8 + (long long)(dy - 1) * a.q.w8);
                    const int row = (vol * 3 + dx) * CIN;
                    tma_load_2d(sa + (uint32_t)(k * CIN * 128), &mx, ux, row, &full[s]);
                }
                tma_load_2d(sb, &mg, (int)u0, vol * COUT, &full[s]);
            }
            for (int j = it > C::kStages ? it - C::kStages : 0; j < it; ++j)
                mb_drain(&full[j % C::kStages], (unsigned)(j / C::kStages) & 1u, a.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = (1u << 4)      // D: FP32
                                       | (1u << 7)    // A: BF16
                                       | (1u << 10)   // B: BF16
                                       | ((uint32_t)(COUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            bool ok = true;
            for (int it = 0; it < nk; ++it) {
                const int s = it % C::kStages;
                if (!mb_wait(&full[s], (unsigned)(it / C::kStages) & 1u, &abort_flag, a.err, 4u, a.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_after();
                const uint32_t sa = sbase + (uint32_t)(s * C::kStage), sb = sa + C::kA;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(tmem, sdesc(sa + (uint32_t)(j * 32), 16, 1024, 2u), sdesc(sb + (uint32_t)(j * 32), 16, 1024, 2u),
                             idesc, (it | j) != 0);
                mma_commit(&empty[s]);
            }
            if (ok && nk > 0) mma_commit(&accf);
            mma_commit(&mma_done);
            mb_drain(&mma_done, 0u, a.err);
        }
    } else if (nk > 0) {   // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int q = warp & 3;
        const bool ok = mb_wait(&accf, 0u, &abort_flag, a.err, 8u, a.wait_ns);
        if (__all_sync(0xFFFFFFFFu, ok)) {
            tc_after();
            const int R = mt * 128 + 32 * q + lane;
            const int t = R / CIN, c = R % CIN;
#pragma unroll
            for (int o0 = 0; o0 < COUT; o0 += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)o0, r);
                if (t < 27) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        atomicAdd(a.dw + ((size_t)(o0 + i) * 27 + t) * CIN + c, __uint_as_float(r[i]));
                }
            }
        }
    }
    __syncwarp();
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols) : "memory");
    }
}

template <int COUT, int CIN>
lsm_status launch_wgrad_tc(const CUtensorMap &mx, const CUtensorMap &mg, WgArgs a, int n, cudaStream_t st)
{
    using C = WgCfg<COUT, CIN>;
    static int occ = 0;
    if (!occ) {
        LSM_CUDA(cudaFuncSetAttribute(k_wgrad_tc<COUT, CIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
        // resident CTAs counted from shared memory, TMEM columns, registers and
        // warps (the occupancy query answers 1 for kernels holding tcgen05)
        cudaFuncAttributes fa;
        LSM_CUDA(cudaFuncGetAttributes(&fa, k_wgrad_tc<COUT, CIN>));
        int dev = 0, smem_sm = 0, rsv = 0;
        LSM_CUDA(cudaGetDevice(&dev));
        LSM_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        LSM_CUDA(cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        const int by_smem = smem_sm / (C::kSmem + (int)fa.sharedSizeBytes + rsv);
        const int by_tmem = 512 / C::kCols;
        const int by_regs = 65536 / (((fa.numRegs + 7) / 8 * 8) * kThreads);
        occ = std::max(1, std::min(std::min(by_smem, by_tmem), std::min(by_regs, 64 / (kThreads / 32))));
    }
    const int target = occ * sm_count();
    a.ksplit = std::max(1, std::min(a.n_chunks, target / (C::kMt * n)));
    const int grid = a.ksplit * C::kMt * n;
    k_wgrad_tc<COUT, CIN><<<grid, kThreads, C::kSmem, st>>>(mx, mg, a);
    count_launch();
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

// dW += the weight gradient of a 3x3x3 layer (cin -> cout) from its input x
// (a channel slice) and its ReLU-masked output gradient gz, on the tensor cores.
lsm_status wgrad_tc(const lsm_vol &gz, const lsm_vol &x, int cin, int cout, float *dw, cudaStream_t st)
{
    const VolIdx v = vidx(x.d, x.h, x.w);
    const L8 q = l8_of(x.d, x.h, x.w);
    const int n = x.n;
    if (q.lq >= (1ll << 30) || (long long)n * 3 * cin > (1 << 20)) return set_arg_error("wgrad: volume too large");
    EncodeTiled enc = encode_fn();
    if (!enc) return set_arg_error("wgrad: cuTensorMapEncodeTiled unavailable");
    unsigned *err = err_word();
    if (!err) return set_cuda_error(cudaErrorMemoryAllocation, "wgrad: error word");
    const size_t nx = (size_t)n * 3 * cin * q.lq, ng = (size_t)n * cout * q.lq;
    __nv_bfloat16 *xt = nullptr;
    LSM_CUDA(dev_malloc((void **)&xt, (nx + ng) * sizeof(__nv_bfloat16) + 256, st));
    __nv_bfloat16 *gt = xt + nx;
    const unsigned gx = (unsigned)((q.lq + 63) / 64);
    k_chmajor<<<dim3(gx, (unsigned)(n * 3)), 256, 0, st>>>((const __nv_bfloat16 *)x.data, x.c_total, x.c_offset, cin,
                                                           v, q, 3, xt);
    count_launch();
    k_chmajor<<<dim3(gx, (unsigned)n), 256, 0, st>>>((const __nv_bfloat16 *)gz.data, gz.c_total, gz.c_offset, cout, v,
                                                     q, 1, gt);
    count_launch();
    cudaError_t ce = cudaGetLastError();
    lsm_status r = LSM_OK;
    CUtensorMap mx, mg;
    const cuuint32_t es[2] = {1, 1};
    const cuuint64_t dx_[2] = {(cuuint64_t)q.lq, (cuuint64_t)n * 3 * cin};
    const cuuint64_t dg_[2] = {(cuuint64_t)q.lq, (cuuint64_t)n * cout};
    const cuuint64_t str[1] = {(cuuint64_t)q.lq * 2};
    const cuuint32_t bx[2] = {64, (cuuint32_t)cin}, bg[2] = {64, (cuuint32_t)cout};
    if (ce != cudaSuccess) {
        r = set_cuda_error(ce, "wgrad: transposition");
    } else if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, xt, dx_, str, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
               enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, gt, dg_, str, bg, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        r = set_arg_error("wgrad: tensor map encoding failed");
    } else {
        WgArgs a;
        a.dw = dw;
        a.q = q;
        const long long u_lo = q.p8 + q.w8 + 1, u_hi = (long long)x.d * q.p8 + (long long)x.h * q.w8 + x.w;
        a.u_first = u_lo / 64 * 64;
        a.n_chunks = (int)((u_hi + 1 - a.u_first + 63) / 64);
        a.ksplit = 1;
        a.err = err;
        a.wait_ns = g_conv_wait_ns;
        switch (cout * 1000 + cin) {
        case 16016: r = launch_wgrad_tc<16, 16>(mx, mg, a, n, st); break;
        case 16032: r = launch_wgrad_tc<16, 32>(mx, mg, a, n, st); break;
        case 32016: r = launch_wgrad_tc<32, 16>(mx, mg, a, n, st); break;
        case 32032: r = launch_wgrad_tc<32, 32>(mx, mg, a, n, st); break;
        case 32064: r = launch_wgrad_tc<32, 64>(mx, mg, a, n, st); break;
        case 64032: r = launch_wgrad_tc<64, 32>(mx, mg, a, n, st); break;
        case 64064: r = launch_wgrad_tc<64, 64>(mx, mg, a, n, st); break;
        case 64128: r = launch_wgrad_tc<64, 128>(mx, mg, a, n, st); break;
        case 128064: r = launch_wgrad_tc<128, 64>(mx, mg, a, n, st); break;
        default: r = set_arg_error("wgrad: unsupported channel configuration");
        }
    }
    cudaFreeAsync(xt, st);
    return r;
}

}  // namespace dn
}  // namespace lsm

namespace lsm {
namespace dn {

void unet_drop_graph(lsm_unet *u)
{
    if (u->gexec) cudaGraphExecDestroy((cudaGraphExec_t)u->gexec);
    u->gexec = nullptr;
    u->g_warm = 0;
    u->g_kernels = 0;
}

lsm_status unet_buffers(lsm_unet *u, int n, int d, int h, int w, cudaStream_t st)
{
    if (u->arena && u->n == n && u->d == d && u->h == h && u->w == w) return LSM_OK;
    LSM_CUDA(cudaStreamSynchronize(st));
    unet_drop_graph(u);                       // it holds the old buffers' addresses
    cudaFree(u->arena);
    cudaFree(u->dmax);
    u->arena = nullptr;
    u->dmax = nullptr;
    size_t off[NBUF], total = 0;
    for (int b = 0; b < NBUF; ++b) {
        const int L = kBufLevel[b];
        off[b] = total;
        total += ((size_t)lsm_vol_bytes(n, d >> L, h >> L, w >> L, kBufCh[b]) + 255) / 256 * 256;
    }
    LSM_CUDA(cudaMalloc(&u->arena, total));
    LSM_CUDA(cudaMalloc(&u->dmax, (size_t)n * 4));
    LSM_CUDA(cudaMemsetAsync(u->arena, 0, total, st));
    for (int b = 0; b < NBUF; ++b) {
        const int L = kBufLevel[b];
        lsm_vol &v = u->vol[b];
        v.data = (char *)u->arena + off[b];
        v.n = n; v.d = d >> L; v.h = h >> L; v.w = w >> L;
        v.c_total = kBufCh[b]; v.c_offset = 0; v.c = kBufCh[b];
    }
    u->n = n; u->d = d; u->h = h; u->w = w;
    return LSM_OK;
}

lsm_vol sub(const lsm_vol &v, int c_offset, int c)
{
    lsm_vol r = v;
    r.c_offset = c_offset;
    r.c = c;
    return r;
}

lsm_status unet_run(lsm_unet *u, const float *dose, const float *rho, float *out, cudaStream_t st)
{
    lsm_vol *V = u->vol;
    const VolIdx v0 = vidx(u->d, u->h, u->w);
    const long long per = (long long)u->d * u->h * u->w;
    const int tk = timer_begin(9, st);
    LSM_CUDA(cudaMemsetAsync(u->dmax, 0, (size_t)u->n * 4, st));
    k_dmax<<<dim3(grid_1d(per) / 4 + 1, std::min(u->n, 64)), 256, 0, st>>>(dose, per, u->n, u->dmax);
    count_launch();
    k_pack_input<<<grid_1d(per * u->n), 256, 0, st>>>(dose, rho, u->dmax, (__nv_bfloat16 *)V[X0].data, u->n, v0);
    count_launch();
    timer_end(tk, st);
    LSM_CUDA(cudaGetLastError());
    auto middle = [&](cudaStream_t s) -> lsm_status {
        lsm_status r = LSM_OK;
        auto conv = [&](int i) -> lsm_status {
            const lsm_vol in = V[kConvIn[i]];
            const lsm_vol o = sub(V[kConvOut[i]], 0, kLayers[i][1]);
            return conv_forward(u->conv[i], &in, &o, 0, s);
        };
        auto pool = [&](int from, int to, int c) -> lsm_status {
            const lsm_vol a = sub(V[from], 0, c);
            return pool_or_up(&a, &V[to], false, s);
        };
        auto up = [&](int from, int to, int c_off) -> lsm_status {
            const lsm_vol b = sub(V[to], c_off, V[from].c);
            return pool_or_up(&V[from], &b, true, s);
        };
        if (!r) r = conv(0);
        if (!r) r = conv(1);
        if (!r) r = pool(S0, P1, kW0);
        if (!r) r = conv(2);
        if (!r) r = conv(3);
        if (!r) r = pool(S1, P2, kW1);
        if (!r) r = conv(4);
        if (!r) r = conv(5);
        if (!r) r = pool(S2, P3, kW2);
        if (!r) r = conv(6);
        if (!r) r = conv(7);
        if (!r) r = up(B3, S2, kW2);
        if (!r) r = conv(8);
        if (!r) r = conv(9);
        if (!r) r = up(D2, S1, kW1);
        if (!r) r = conv(10);
        if (!r) r = conv(11);
        if (!r) r = up(D1, S0, kW0);
        if (!r) r = conv(12);
        if (!r) r = conv(13);
        return r;
    };
    lsm_status rc = LSM_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LSM_CUDA(cudaStreamIsCapturing(st, &cap));
    if (timing_enabled() || u->g_warm != 1 || cap != cudaStreamCaptureStatusNone) {
        // per-kernel timers need the direct launches; the first pass on new
        // buffers runs directly too (one-time attribute and table set-up); a
        // caller capturing its own graph gets the layers as its own nodes
        rc = middle(st);
        if (!rc && u->g_warm == 0) u->g_warm = 1;
    } else {
        if (!u->gexec) {
            cudaStream_t cs = nullptr;
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            const int64_t c0 = lsm_launch_count();
            cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            lsm_status r = LSM_OK;
            if (e == cudaSuccess) {
                r = middle(cs);
                e = cudaStreamEndCapture(cs, &g);
            }
            const int64_t captured = lsm_launch_count() - c0;
            add_launches(-captured);           // counted when replayed
            if (e == cudaSuccess && !r && g) e = cudaGraphInstantiate(&ex, g, 0);
            if (g) cudaGraphDestroy(g);
            if (cs) cudaStreamDestroy(cs);
            if (e == cudaSuccess && !r && ex) {
                u->gexec = ex;
                u->g_kernels = captured;
            } else {
                if (ex) cudaGraphExecDestroy(ex);
                cudaGetLastError();
                u->g_warm = -1;                // capture failed: direct launches for these buffers
            }
        }
        if (u->gexec) {
            LSM_CUDA(cudaGraphLaunch((cudaGraphExec_t)u->gexec, st));
            add_launches(u->g_kernels);
        } else {
            rc = middle(st);
        }
    }
    if (rc || !out) return rc;
    const int th = timer_begin(9, st);
    k_head<<<grid_1d(per * u->n), 256, 0, st>>>((const __nv_bfloat16 *)V[D0].data, V[D0].c_total, u->head, dose,
                                                u->dmax, out, u->n, v0);
    count_launch();
    timer_end(th, st);
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

}  // namespace dn
}  // namespace lsm

using namespace lsm;

extern "C" {

int64_t lsm_vol_bytes(int32_t n, int32_t d, int32_t h, int32_t w, int32_t c_total)
{
    if (n < 1 || d < 1 || h < 1 || w < 1 || c_total < 1) return 0;
    return (int64_t)n * (d + 2) * (int64_t)(h + 2) * (w + 2) * c_total * 2;
}

lsm_status lsm_conv3d_create(int32_t c_in, int32_t c_out, int32_t relu, const float *weight, const float *bias,
                             lsm_conv3d **out, lsm_stream stream)
{
    return dn::conv_create(c_in, c_out, relu, weight, bias, out, (cudaStream_t)stream);
}

void lsm_conv3d_destroy(lsm_conv3d *conv) { dn::conv_destroy(conv); }

lsm_status lsm_conv3d_forward(const lsm_conv3d *conv, const lsm_vol *in, const lsm_vol *out, int32_t ctas_per_sm,
                              lsm_stream stream)
{
    return dn::conv_forward(conv, in, out, ctas_per_sm, (cudaStream_t)stream);
}

lsm_status lsm_pool3d(const lsm_vol *in, const lsm_vol *out, lsm_stream stream)
{
    return dn::pool_or_up(in, out, false, (cudaStream_t)stream);
}

lsm_status lsm_upsample3d(const lsm_vol *in, const lsm_vol *out, lsm_stream stream)
{
    return dn::pool_or_up(in, out, true, (cudaStream_t)stream);
}

int64_t lsm_unet_param_count(void) { return dn::param_count(); }

lsm_status lsm_unet_create(const float *params, int64_t n_params, lsm_unet **out, lsm_stream stream)
{
    if (!params || !out) return set_arg_error("lsm_unet_create: NULL argument");
    if (n_params != dn::param_count()) return set_arg_error("lsm_unet_create: wrong parameter count");
    lsm_unet *u = (lsm_unet *)calloc(1, sizeof(lsm_unet));
    if (!u) return set_arg_error("lsm_unet_create: out of host memory");
    const cudaStream_t st = (cudaStream_t)stream;
    lsm_status rc = LSM_OK;
    cudaError_t e = cudaMalloc(&u->params, (size_t)n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(u->params, params, (size_t)n_params * sizeof(float),
                                              cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = set_cuda_error(e, "lsm_unet_create");
    u->head = u->params ? u->params + dn::layer_offset(14) : nullptr;
    for (int i = 0; i < 14 && !rc; ++i) {
        rc = dn::conv_alloc(dn::kLayers[i][0], dn::kLayers[i][1], 1, &u->conv[i]);
        if (!rc) rc = dn::pack_layer(u, i, st);
    }
    if (!rc && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = set_cuda_error(e, "lsm_unet_create");
    if (rc) {
        lsm_unet_destroy(u);
        return rc;
    }
    *out = u;
    return LSM_OK;
}

void lsm_unet_destroy(lsm_unet *u)
{
    if (!u) return;
    cudaDeviceSynchronize();
    dn::unet_drop_graph(u);
    for (int i = 0; i < 14; ++i) dn::conv_destroy(u->conv[i]);
    dn::train_free(u->train);
    cudaFree(u->params);
    cudaFree(u->arena);
    cudaFree(u->dmax);
    cudaFree(u->io);
    free(u);
}

lsm_status lsm_unet_forward(lsm_unet *u, int32_t n, int32_t d, int32_t h, int32_t w, const float *dose,
                            const float *rho, float *out, lsm_mem mem, lsm_stream stream)
{
    if (!u || !dose || !rho || !out) return set_arg_error("lsm_unet_forward: NULL argument");
    if (n < 1 || d < 8 || h < 8 || w < 8 || d % 8 || h % 8 || w % 8)
        return set_arg_error("lsm_unet_forward: n >= 1 and d, h, w positive multiples of 8");
    const cudaStream_t st = (cudaStream_t)stream;
    lsm_status rc = dn::unet_buffers(u, n, d, h, w, st);
    if (rc) return rc;
    const size_t nv = (size_t)n * d * h * w;
    if (mem == LSM_MEM_DEVICE) return dn::unet_run(u, dose, rho, out, st);
    if (u->io_cap < nv) {
        LSM_CUDA(cudaStreamSynchronize(st));
        cudaFree(u->io);
        u->io = nullptr;
        u->io_cap = 0;
        LSM_CUDA(cudaMalloc(&u->io, 3 * nv * sizeof(float)));
        u->io_cap = nv;
    }
    LSM_CUDA(cudaMemcpyAsync(u->io, dose, nv * 4, cudaMemcpyHostToDevice, st));
    LSM_CUDA(cudaMemcpyAsync(u->io + nv, rho, nv * 4, cudaMemcpyHostToDevice, st));
    rc = dn::unet_run(u, u->io, u->io + nv, u->io + 2 * nv, st);
    if (rc) return rc;
    LSM_CUDA(cudaMemcpyAsync(out, u->io + 2 * nv, nv * 4, cudaMemcpyDeviceToHost, st));
    unsigned err = 0;
    LSM_CUDA(cudaMemcpyAsync(&err, dn::err_word(), 4, cudaMemcpyDeviceToHost, st));
    LSM_CUDA(cudaStreamSynchronize(st));
    if (err) {
        cudaMemsetAsync(dn::err_word(), 0, 4, st);
        set_arg_error("lsm_unet_forward: a tensor-core pipeline wait timed out");
        return LSM_ERR_TIMEOUT;
    }
    return LSM_OK;
}

lsm_status lsm_unet_activation(const lsm_unet *u, int32_t layer, void *dst, lsm_mem mem, lsm_stream stream)
{
    if (!u || !dst) return set_arg_error("lsm_unet_activation: NULL argument");
    if (layer < 0 || layer >= 14) return set_arg_error("lsm_unet_activation: layer in 0..13");
    if (!u->arena) return set_arg_error("lsm_unet_activation: no forward call yet");
    const cudaStream_t st = (cudaStream_t)stream;
    const lsm_vol &v = u->vol[dn::kConvOut[layer]];
    const int c = dn::kLayers[layer][1];
    const size_t count = (size_t)v.n * v.d * v.h * v.w * c;
    void *tmp = dst;
    if (mem == LSM_MEM_HOST) LSM_CUDA(cudaMalloc(&tmp, count * 2));
    dn::k_extract<<<dn::grid_1d((long long)count), 256, 0, st>>>((const __nv_bfloat16 *)v.data, v.c_total, 0, c,
                                                                 (__nv_bfloat16 *)tmp, v.n, dn::vidx(v.d, v.h, v.w));
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem == LSM_MEM_HOST) {
        e = cudaMemcpyAsync(dst, tmp, count * 2, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(tmp);
    }
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_unet_activation");
    return LSM_OK;
}

}  // extern "C"
