// psl_build.cu -- PSR -> PSL conversion, sampling areas and Eq. 3 counts on the GPU.
//
// Sec. 2.1.1 (Eq. 1-2 and the four conversion steps), Sec. 2.1.2 (sampling
// areas, Fig. 3), step S2 (Eq. 3) and the loop order of Sec. 2.1.3.
//
// Everything here is FP64 and this translation unit is compiled with
// -fmad=false: each per-PSL value is the correctly rounded result of one fixed
// sequence of IEEE operations, and every sum runs in one fixed order (sums
// over a block's PSLs in the 32-way order of warp_sum32, the others
// sequentially in loop order), so the integer counts that Eq. 3 produces do
// not depend on thread scheduling. The integerisation is largest-remainder (Hamilton) with ties to
// the lower loop index; integer sums use 64-bit atomics (exact, any order).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "handles.cuh"

namespace lsm {
namespace {

__device__ void ring_interp(double r, int n_r, double dr, int *r0, double *l0, int *inside)
{
    *inside = 1;
    if (r >= (double)n_r * dr) { *r0 = n_r - 1; *l0 = 1.0; *inside = 0; return; }
    double t = r / dr - 0.5;
    if (t <= 0.0) { *r0 = 0; *l0 = 1.0; return; }
    if (t >= (double)(n_r - 1)) { *r0 = n_r - 1; *l0 = 1.0; return; }
    int i = (int)floor(t);
    *r0 = i;
    *l0 = 1.0 - (t - (double)i);
}

__device__ __forceinline__ double psl_radius(int ix, int iy, int n_r, double p)
{
    double xc = ((double)(ix - n_r) + 0.5) * p;
    double yc = ((double)(iy - n_r) + 0.5) * p;
    return sqrt(xc * xc + yc * yc);
}

struct Geom {
    const double *jaws;
    int n_beams;
    double z_phsp, sad, z_jaw_x, z_jaw_y;
};

// Sampling areas of beam b on the phase-space plane: a[0..3] primary, a[4..7]
// scatter/electrons (xa, xb, ya, yb).
__device__ __forceinline__ void beam_area(const Geom &G, int b, double a[8])
{
    const double x1 = G.jaws[4 * b], x2 = G.jaws[4 * b + 1], y1 = G.jaws[4 * b + 2], y2 = G.jaws[4 * b + 3];
    const double k = G.z_phsp / G.sad;                // primary: opening scaled to the plane
    a[0] = x1 * k; a[1] = x2 * k; a[2] = y1 * k; a[3] = y2 * k;
    const double cx = 0.5 * (x1 + x2), cy = 0.5 * (y1 + y2);
    const double fx = (G.sad - G.z_phsp) / (G.sad - G.z_jaw_x), fy = (G.sad - G.z_phsp) / (G.sad - G.z_jaw_y);
    const double kx = G.z_jaw_x / G.sad, ky = G.z_jaw_y / G.sad;
    a[4] = cx + (x1 * kx - cx) * fx;                  // scatter/electrons: back projection
    a[5] = cx + (x2 * kx - cx) * fx;
    a[6] = cy + (y1 * ky - cy) * fy;
    a[7] = cy + (y2 * ky - cy) * fy;
}

// Areas (and the single-precision jaw limits in the jaw planes for the
// rejection test), one thread per beam.
__device__ __forceinline__ void write_areas(const Geom &G, int b, double *__restrict__ area,
                                            float *__restrict__ jaws_f)
{
    double a[8];
    beam_area(G, b, a);
    for (int k = 0; k < 8; ++k) area[8 * b + k] = a[k];
    const double x1 = G.jaws[4 * b], x2 = G.jaws[4 * b + 1], y1 = G.jaws[4 * b + 2], y2 = G.jaws[4 * b + 3];
    jaws_f[4 * b + 0] = (float)(y1 * G.z_jaw_y / G.sad);
    jaws_f[4 * b + 1] = (float)(y2 * G.z_jaw_y / G.sad);
    jaws_f[4 * b + 2] = (float)(x1 * G.z_jaw_x / G.sad);
    jaws_f[4 * b + 3] = (float)(x2 * G.z_jaw_x / G.sad);
}

// PSL inclusion of cell i = (beam, class, PSL): positive-area overlap with the
// class's sampling area.
__device__ __forceinline__ void incl_cell(const Geom &G, int n_r, double p, int64_t i, uint8_t *__restrict__ incl)
{
    const int nxy = 2 * n_r, npsl = nxy * nxy;
    const int j = (int)(i % npsl), bc = (int)(i / npsl);
    const int iy = j / nxy, ix = j % nxy;
    double area[8];
    beam_area(G, bc >> 1, area);
    const double *a = area + 4 * (bc & 1);
    const double xl = (double)(ix - n_r) * p, xh = (double)(ix - n_r + 1) * p;
    const double yl = (double)(iy - n_r) * p, yh = (double)(iy - n_r + 1) * p;
    incl[i] = (uint8_t)(xh > a[0] && xl < a[1] && yh > a[2] && yl < a[3]);
}

// The plan's sums over the PSLs of a block (step 4's raw total, Eq. 3's
// partial denominators, a basis run's denominator) in one fixed order, the
// oracle's or_sum32: lane l of one warp adds x[l], x[l + 32], ... in index
// order from 0.0, then an xor butterfly over the lanes (offsets 16, 8, 4, 2,
// 1; both lanes of a pair form the same IEEE sum, so lane 0 ends with the
// halving order). Excluded elements (mask 0) contribute +0.0. All 32 lanes
// call it; lane 0's result is the sum in that order (the other lanes hold
// the same terms added in other orders). A sequential FP64 sum of a block's
// 400 PSLs was a chain of 400 dependent adds on the B300's narrow FP64
// pipe: the plan build 0.109 -> 0.080 ms.
__device__ __forceinline__ double warp_sum32(const double *x, const uint8_t *mask, int n)
{
    const int lane = threadIdx.x & 31;
    double a = 0.0;
    for (int j = lane; j < n; j += 32) a += (mask && !mask[j]) ? 0.0 : x[j];
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// Steps 1-4 per (sub-source, energy bin) block: one CTA per block.
__device__ __forceinline__ void psl_weights_block(int blk, const double *__restrict__ w, int n_e, int n_r, double dr,
                                                  double *__restrict__ wpsl, double *__restrict__ block_scale,
                                                  int32_t *__restrict__ tag_r0, double *__restrict__ tag_l0)
{
    const int nxy = 2 * n_r, npsl = nxy * nxy;
    const double *W = w + (size_t)blk * n_r;
    double *out = wpsl + (size_t)blk * npsl;
    extern __shared__ double sraw_v[];
    // the ring densities W_R / dr, one division per ring instead of two per
    // PSL (the same correctly rounded quotients)
    __shared__ double s_wd[32];
    if ((int)threadIdx.x < n_r) s_wd[threadIdx.x] = W[threadIdx.x] / dr;
    __syncthreads();
    for (int j = threadIdx.x; j < npsl; j += blockDim.x) {
        const int iy = j / nxy, ix = j % nxy;
        const double r = psl_radius(ix, iy, n_r, dr);                    // step 1
        int r0, in;
        double l0;
        ring_interp(r, n_r, dr, &r0, &l0, &in);
        double dens = 0.0;                                               // step 2
        if (in) {
            dens = l0 * s_wd[r0];
            if (l0 < 1.0) dens += (1.0 - l0) * s_wd[r0 + 1];
        }
        out[j] = dens / (2.0 * kPiD * r);                               // step 3
        sraw_v[j] = out[j];
        if (blk == 0) {
            tag_r0[j] = r0;
            tag_l0[j] = in ? l0 : 0.0;
        }
    }
    __syncthreads();
    __shared__ double s_scale;
    if (threadIdx.x < 32) {                                              // step 4
        const double sraw = warp_sum32(sraw_v, nullptr, npsl);
        if (threadIdx.x == 0) {
            double sR = 0.0;
            for (int R = 0; R < n_r; ++R) sR += W[R];
            s_scale = sraw > 0.0 ? sR / sraw : 0.0;
            block_scale[blk] = s_scale;
        }
    }
    __syncthreads();
    const double sc = s_scale;
    for (int j = threadIdx.x; j < npsl; j += blockDim.x) out[j] = out[j] * sc;
}

__device__ __forceinline__ void dir_tables_one(const double *__restrict__ mc, const double *__restrict__ mmu,
                                               const double *__restrict__ msa, const double *__restrict__ msb,
                                               const double *__restrict__ esa, const double *__restrict__ esb, int i,
                                               unsigned long long *__restrict__ thr, float4 *__restrict__ mix,
                                               float2 *__restrict__ esig);

struct SetupArgs {
    const double *w;
    int n_e, n_r;
    double dr;
    double *wpsl, *block_scale;
    int32_t *tag_r0;
    double *tag_l0;
    Geom G;
    double *area;
    float *jaws_f;
    uint8_t *incl;
    int n_incl_blocks;
    const double *mc, *mmu, *msa, *msb, *esa, *esb;
    int nes;
    unsigned long long *thr;
    float4 *mix;
    float2 *esig;
};

// One launch for the independent set-up work of a plan, by block: the PSL
// weights of each (sub-source, energy) block, the sampling areas and PSL
// inclusion of every beam, and the direction tables.
__global__ void k_setup(SetupArgs A)
{
    const int nw = 3 * A.n_e;
    int blk = blockIdx.x;
    if (blk < nw) {
        psl_weights_block(blk, A.w, A.n_e, A.n_r, A.dr, A.wpsl, A.block_scale, A.tag_r0, A.tag_l0);
        return;
    }
    blk -= nw;
    if (blk < A.n_incl_blocks) {
        const int npsl = 4 * A.n_r * A.n_r;
        const int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
        if (blk == 0 && (int)threadIdx.x < A.G.n_beams) write_areas(A.G, threadIdx.x, A.area, A.jaws_f);
        if (i < (int64_t)A.G.n_beams * 2 * npsl) incl_cell(A.G, A.n_r, A.dr, i, A.incl);
        return;
    }
    blk -= A.n_incl_blocks;
    const int i = blk * blockDim.x + threadIdx.x;
    if (i < A.nes) dir_tables_one(A.mc, A.mmu, A.msa, A.msb, A.esa, A.esb, i, A.thr, A.mix, A.esig);
}

// ------------------------------------------------ whole-source plan (Eq. 3) --

// partial sum of included weights per (beam, sub-source, energy) in the
// warp_sum32 order; one CTA per block stages the values through shared memory
__global__ void k_eq3_parts(const double *__restrict__ wpsl, const uint8_t *__restrict__ incl,
                            int n_beams, int n_e, int npsl, double *__restrict__ parts)
{
    extern __shared__ double sv[];
    const int i = blockIdx.x;
    const int b = i / (3 * n_e), s = (i / n_e) % 3, e = i % n_e;
    const uint8_t *inc = incl + (size_t)(b * 2 + (s ? 1 : 0)) * npsl;
    const double *W = wpsl + ((size_t)s * n_e + e) * npsl;
    for (int j = threadIdx.x; j < npsl; j += blockDim.x) sv[j] = W[j];
    __syncthreads();
    if (threadIdx.x < 32) {
        const double part = warp_sum32(sv, inc, npsl);
        if (threadIdx.x == 0) parts[i] = part;
    }
}

// Eq. 3 floors. The denominator is the sequential sum of the partial sums
// in (beam, sub-source, energy) order, formed by every block (block 0 stores it).
__global__ void k_eq3_floor(const double *__restrict__ wpsl, const uint8_t *__restrict__ incl,
                            int n_e, int npsl, int64_t ncell, int64_t n_hist, const double *__restrict__ parts,
                            int n_parts, double *__restrict__ denom, int64_t *__restrict__ count,
                            double *__restrict__ rem, unsigned long long *__restrict__ floor_sum)
{
    __shared__ double s_D;
    if (threadIdx.x == 0) {
        double D = 0.0;
        for (int k = 0; k < n_parts; ++k) D += parts[k];
        s_D = D;
        if (blockIdx.x == 0) *denom = D;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long f = 0;
    if (i < ncell) {
        const int j = (int)(i % npsl);
        const int64_t bse = i / npsl;
        const int e = (int)(bse % n_e), s = (int)((bse / n_e) % 3), b = (int)(bse / (3 * n_e));
        const double D = s_D;
        const bool inc = incl[(size_t)(b * 2 + (s ? 1 : 0)) * npsl + j] != 0;
        const double q = (inc && D > 0.0) ? ((double)n_hist * wpsl[((size_t)s * n_e + e) * npsl + j]) / D
                                          : 0.0;
        const double fl = floor(q);
        f = (long long)fl;
        count[i] = f;
        rem[i] = q - fl;
    }
    // block-level reduction of the floors, then one atomic per block
    __shared__ unsigned long long red[32];
    unsigned long long v = warp_sum_u64((unsigned long long)f);
    if (lane_id() == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
        t = warp_sum_u64(t);
        if (threadIdx.x == 0) atomicAdd(floor_sum, t);
    }
}

// Largest remainders: the `left` cells of highest remainder, ties to the
// lower loop index, get one more particle. Remainders are finite and >= 0, so
// they order exactly as their IEEE bit patterns read as unsigned integers. One
// CTA finds the left-th largest key by an 8-pass most-significant-digit radix
// select (256-bin histograms of the keys that match the digits chosen so far),
// then adds one to every cell with a larger key and to the first `need` cells,
// in loop order, whose key equals it.
__device__ void eq3_select_apply(const double *__restrict__ rem, int64_t n, long long left, int64_t *__restrict__ count)
{
    const unsigned long long *key = reinterpret_cast<const unsigned long long *>(rem);
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_pre;
    __shared__ long long s_k;
    __shared__ int s_all;     // every key of the chosen bin is taken: the selection is the keys >= s_pre
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) { s_pre = 0ull; s_k = left; s_all = 0; }
    unsigned long long mask = 0ull;
    for (int shift = 56; shift >= 0; shift -= 8) {
        if (tid < 256) hist[tid] = 0u;
        __syncthreads();
        const unsigned long long pre = s_pre;
        for (int64_t i = tid; i < n; i += blockDim.x) {
            const unsigned long long k = key[i];
            if ((k & mask) == pre) atomicAdd(&hist[(unsigned)(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (wid == 0) {
            // lane l holds bins [8 l, 8 l + 8); suffix sums from the top bin down
            unsigned c[8], loc = 0;
            for (int j = 0; j < 8; ++j) { c[j] = hist[8 * lane + j]; loc += c[j]; }
            unsigned suf = loc;                      // inclusive suffix over lanes >= lane
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_down_sync(0xffffffffu, suf, o);
                if (lane + o < 32) suf += v;
            }
            const long long k = s_k;
            long long above = (long long)(suf - loc); // keys in bins above this lane's
            int found = -1;
            long long rest = 0;
            unsigned cf = 0;
            for (int j = 7; j >= 0; --j) {
                if (found < 0 && above < k && above + (long long)c[j] >= k) {
                    found = 8 * lane + j;
                    rest = k - above;
                    cf = c[j];
                }
                above += c[j];
            }
            const unsigned hit = __ballot_sync(0xffffffffu, found >= 0);
            const int src = __ffs(hit) - 1;
            const int bin = __shfl_sync(0xffffffffu, found, src);
            const long long kk = __shfl_sync(0xffffffffu, rest, src);
            const unsigned cb = __shfl_sync(0xffffffffu, cf, src);
            if (lane == 0) {
                s_pre = pre | ((unsigned long long)bin << shift);
                s_k = kk;
                // the bin's keys are all taken: keys above the prefix were taken
                // by earlier digits, the rest lie below it
                if ((long long)cb == kk) s_all = 1;
            }
        }
        mask |= 255ull << shift;
        __syncthreads();
        if (s_all) break;
    }
    if (s_all) {
        const unsigned long long thr = s_pre;
        for (int64_t i = tid; i < n; i += blockDim.x)
            if (key[i] >= thr) count[i] += 1;
        return;
    }
    const unsigned long long v = s_pre;             // the left-th largest key
    const long long need = s_k;                      // cells with key == v that get one more
    // scan of the (key == v) flags in loop order over per-thread segments
    const int T = blockDim.x;
    const int64_t seg = (n + T - 1) / T;
    const int64_t a = (int64_t)tid * seg, bnd = a + seg < n ? a + seg : n;
    long long s = 0;
    for (int64_t i = a; i < bnd; ++i) s += key[i] == v ? 1 : 0;
    __shared__ long long wsum[32];
    long long inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (T >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    long long run = inc - s + (wid ? wsum[wid - 1] : 0);
    for (int64_t i = a; i < bnd; ++i) {
        const unsigned long long k = key[i];
        if (k > v) count[i] += 1;
        else if (k == v) { if (run < need) count[i] += 1; ++run; }
    }
}

__device__ void scan_counts_block(const int64_t *__restrict__ count, int64_t n, int64_t *__restrict__ cstart,
                                  int64_t *__restrict__ eidx, int64_t *__restrict__ start, int64_t *__restrict__ res);

// One CTA: the largest remainders, then (the counts final) the exclusive
// scans of the counts that place the plan's entries, in one launch.
__global__ void __launch_bounds__(1024) k_eq3_select(const double *__restrict__ rem, int64_t n, int64_t n_hist,
                                                     const unsigned long long *__restrict__ floor_sum,
                                                     const double *__restrict__ denom, int64_t *__restrict__ count,
                                                     int64_t *__restrict__ cstart, int64_t *__restrict__ eidx,
                                                     int64_t *__restrict__ start, int64_t *__restrict__ res)
{
    // an empty sampling area (denominator 0) distributes nothing
    const long long left = (*denom > 0.0 ? n_hist : 0) - (long long)(*floor_sum);
    if (left > 0) eq3_select_apply(rem, n, left, count);      // uniform over the block
    __syncthreads();
    scan_counts_block(count, n, cstart, eidx, start, res);
}

// ------------------------------------------------- per-PSR basis-run plans --

// One CTA per (PSR k, beam b): weights of PSR k's share, Eq. 3 within the run.
__global__ void k_psr_counts(const double *__restrict__ w, const double *__restrict__ block_scale,
                             const uint8_t *__restrict__ incl, const int64_t *__restrict__ n_k,
                             int n_e, int n_r, double dr, int n_beams,
                             int64_t *__restrict__ count, double *__restrict__ dkb)
{
    extern __shared__ double sm[];
    const int nxy = 2 * n_r, npsl = nxy * nxy;
    double *q = sm;                 // [npsl]
    double *rm = sm + npsl;         // [npsl]
    long long *fl = (long long *)(sm + 2 * npsl);
    __shared__ double s_D;
    __shared__ long long s_left;
    const int kb = blockIdx.x;
    const int k = kb / n_beams, b = kb % n_beams;
    const int s = k / (n_e * n_r), e = (k / n_r) % n_e, R = k % n_r;
    const double *W = w + ((size_t)s * n_e + e) * n_r;
    const double scale = block_scale[s * n_e + e];
    const uint8_t *inc = incl + (size_t)(b * 2 + (s ? 1 : 0)) * npsl;
    for (int j = threadIdx.x; j < npsl; j += blockDim.x) {
        const int iy = j / nxy, ix = j % nxy;
        const double r = psl_radius(ix, iy, n_r, dr);
        int r0, in;
        double l0;
        ring_interp(r, n_r, dr, &r0, &l0, &in);
        double dk = 0.0;
        if (in) {
            if (r0 == R) dk = l0 * (W[R] / dr);
            else if (r0 + 1 == R && l0 < 1.0) dk = (1.0 - l0) * (W[R] / dr);
        }
        q[j] = (dk / (2.0 * kPiD * r)) * scale;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const double D = warp_sum32(q, inc, npsl);
        if (threadIdx.x == 0) {
            s_D = D;
            dkb[kb] = D;
        }
    }
    __syncthreads();
    const double D = s_D;
    const int64_t nk = n_k[k];
    for (int j = threadIdx.x; j < npsl; j += blockDim.x) {
        const double qq = (inc[j] && D > 0.0) ? ((double)nk * q[j]) / D : 0.0;
        const double f = floor(qq);
        fl[j] = (long long)f;
        rm[j] = qq - f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long sfl = 0;
        for (int j = 0; j < npsl; ++j) sfl += fl[j];
        s_left = (D > 0.0 ? nk : 0) - sfl;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < npsl; j += blockDim.x) {
        const double rj = rm[j];
        int rank = 0;
        for (int t = 0; t < npsl; ++t) rank += (rm[t] > rj) || (rm[t] == rj && t < j);
        count[(size_t)kb * npsl + j] = fl[j] + (rank < s_left ? 1 : 0);
    }
}

// ------------------------------------------------------ scans and entries --

// Plan prefix of the counts (cstart) and entry index of the non-empty cells
// (eidx) in one pass of one CTA, and the plan end start[n_ent] = total;
// (n_ent, total) also go to res[0..1] for the host.
__device__ void scan_counts_block(const int64_t *__restrict__ count, int64_t n, int64_t *__restrict__ cstart,
                                  int64_t *__restrict__ eidx, int64_t *__restrict__ start, int64_t *__restrict__ res)
{
    const int T = blockDim.x;
    const int64_t seg = (n + T - 1) / T;
    const int64_t a = (int64_t)threadIdx.x * seg, bnd = a + seg < n ? a + seg : n;
    long long s = 0, z = 0;
    for (int64_t i = a; i < bnd; ++i) { const long long c = count[i]; s += c; z += c > 0 ? 1 : 0; }
    __shared__ long long ws[32], wz[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long is = s, iz = z;
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, is, o), u = __shfl_up_sync(0xffffffffu, iz, o);
        if (lane >= o) { is += v; iz += u; }
    }
    if (lane == 31) { ws[wid] = is; wz[wid] = iz; }
    __syncthreads();
    if (wid == 0) {
        long long x = lane < (T >> 5) ? ws[lane] : 0, y = lane < (T >> 5) ? wz[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long v = __shfl_up_sync(0xffffffffu, x, o), u = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) { x += v; y += u; }
        }
        ws[lane] = x;
        wz[lane] = y;
        if (lane == 31) { cstart[n] = x; eidx[n] = y; start[y] = x; res[0] = y; res[1] = x; }
    }
    __syncthreads();
    long long rs = is - s + (wid ? ws[wid - 1] : 0), rz = iz - z + (wid ? wz[wid - 1] : 0);
    for (int64_t i = a; i < bnd; ++i) {
        const long long c = count[i];
        cstart[i] = rs;
        eidx[i] = rz;
        rs += c;
        rz += c > 0 ? 1 : 0;
    }
}

__global__ void k_scan_counts(const int64_t *__restrict__ count, int64_t n, int64_t *__restrict__ cstart,
                              int64_t *__restrict__ eidx, int64_t *__restrict__ start, int64_t *__restrict__ res)
{
    scan_counts_block(count, n, cstart, eidx, start, res);
}


__device__ unsigned long long thresh32(double p)
{
    double t = floor(p * 4294967296.0);
    if (t < 0.0) t = 0.0;
    if (t > 4294967296.0) t = 4294967296.0;
    return (unsigned long long)t;
}

// write the entry table; cells in loop order (whole-source: [b][s][e][y][x],
// per-PSR: [k][b][y][x])
__global__ void k_entries(const int64_t *__restrict__ count, const int64_t *__restrict__ cstart,
                          const int64_t *__restrict__ eidx, int64_t ncell, int per_psr, int n_beams,
                          int n_e, int n_r, const double *__restrict__ w,
                          const int32_t *__restrict__ tag_r0, const double *__restrict__ tag_l0,
                          const double *__restrict__ dkb, const int64_t *__restrict__ n_k,
                          int64_t *__restrict__ start, EntryRec *__restrict__ ent,
                          double *__restrict__ escale)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell || count[i] <= 0) return;
    const int nxy = 2 * n_r, npsl = nxy * nxy;
    const int j = (int)(i % npsl);
    const int64_t o = i / npsl;
    int b, s, e, fixed = -1;
    double sc = 0.0;
    if (per_psr) {
        const int k = (int)(o / n_beams);
        b = (int)(o % n_beams);
        s = k / (n_e * n_r); e = (k / n_r) % n_e;
        fixed = k % n_r;
        sc = dkb[k * n_beams + b] / (double)n_k[k];
    } else {
        e = (int)(o % n_e); s = (int)((o / n_e) % 3); b = (int)(o / (3 * n_e));
    }
    EntryRec r;
    r.ix = (uint16_t)(j % nxy);
    r.iy = (uint16_t)(j / nxy);
    r.beam = (uint8_t)b;
    r.stype = (uint8_t)s;
    r.ebin = (uint16_t)e;
    r.pad = 0;
    const int r0 = tag_r0[j];
    const double l0 = tag_l0[j];
    r.r0 = (uint8_t)r0;
    r.thr = 0;
    if (fixed < 0) {
        fixed = r0;
        if (l0 < 1.0 && r0 + 1 < n_r) {
            const double *W = w + ((size_t)s * n_e + e) * n_r;
            const double a0 = l0 * W[r0], a1 = (1.0 - l0) * W[r0 + 1];
            const double p0 = (a0 + a1) > 0.0 ? a0 / (a0 + a1) : 1.0;
            const unsigned long long T = thresh32(p0);
            if (T == 0ull) fixed = r0 + 1;
            else if (T >= 4294967296ull) fixed = r0;
            else { fixed = -1; r.thr = (uint32_t)T; }
        }
    }
    r.fixed_ring = (int16_t)fixed;
    const int64_t q = eidx[i];
    ent[q] = r;
    start[q] = cstart[i];
    escale[q] = sc;
}


// scatter-mixture component thresholds and single-precision direction tables
__device__ __forceinline__ void dir_tables_one(const double *__restrict__ mc, const double *__restrict__ mmu,
                                               const double *__restrict__ msa, const double *__restrict__ msb,
                                               const double *__restrict__ esa, const double *__restrict__ esb, int i,
                                               unsigned long long *__restrict__ thr, float4 *__restrict__ mix,
                                               float2 *__restrict__ esig)
{
    const double *c = mc + 3 * i;
    const double tot = c[0] + c[1] + c[2];
    thr[2 * i] = thresh32(c[0] / tot);
    thr[2 * i + 1] = thresh32((c[0] + c[1]) / tot);
    for (int k = 0; k < 3; ++k)
        mix[3 * i + k] = make_float4((float)mmu[3 * i + k], (float)msa[3 * i + k],
                                     (float)msb[3 * i + k], 0.0f);
    esig[i] = make_float2((float)esa[i], (float)esb[i]);
}

bool finite_nonneg(const double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!(a[i] >= 0.0) || !isfinite(a[i])) return false;
    return true;
}

}  // namespace

lsm_status free_psl(lsm_psl *p);

namespace {
// Pinned 32-byte result slots, one per plan: the build's final copy lands
// there asynchronously. Taken from 1024-slot slabs that are never released.
std::mutex g_slot_m;
std::vector<int64_t *> g_free_slots;

int64_t *take_slot()
{
    std::lock_guard<std::mutex> lk(g_slot_m);
    if (g_free_slots.empty()) {
        int64_t *slab = nullptr;
        if (cudaMallocHost((void **)&slab, 1024 * 32) != cudaSuccess) return nullptr;
        for (int i = 1023; i >= 0; --i) g_free_slots.push_back(slab + 4 * i);
    }
    int64_t *p = g_free_slots.back();
    g_free_slots.pop_back();
    return p;
}

void give_slot(int64_t *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_slot_m);
    g_free_slots.push_back(p);
}
}  // namespace

// Wait for the build's results and check them (once).
lsm_status resolve_psl(lsm_psl *P)
{
    if (P->resolved) {
        if (P->empty) return set_arg_error("lsm_build_psl: the sampling areas hold no PSL with non-zero weight");
        return LSM_OK;
    }
    LSM_CUDA(cudaEventSynchronize((cudaEvent_t)P->done));
    const int64_t *res = P->h_res;
    const int64_t n_ent = res[2], total = res[3];
    P->resolved = 1;
    if (n_ent < 1 || total < 1) {
        P->empty = 1;
        return set_arg_error("lsm_build_psl: the sampling areas hold no PSL with non-zero weight");
    }
    if (!P->per_psr) memcpy(&P->denom, &res[0], 8);
    P->n_ent = n_ent;
    P->plan_size = total;
    return LSM_OK;
}

// Validation of a PSR model (the ranges stated at lsm_psr_model).
static lsm_status validate_model(const lsm_psr_model *M)
{
    if (M->n_e < 1 || M->n_e > 64 || M->n_r < 1 || M->n_r > 32)
        return set_arg_error("lsm_model_create: need 1 <= n_e <= 64 and 1 <= n_r <= 32");
    if (!(M->dr > 0) || !(M->z_phsp > 0) || !(M->sigma_s >= 0) || !isfinite(M->sigma_s) || !isfinite(M->dr) ||
        !isfinite(M->z_phsp))
        return set_arg_error("lsm_model_create: dr, z_phsp must be > 0 and sigma_s >= 0");
    for (int s = 0; s < 3; ++s)
        if (!(M->de[s] > 0) || !isfinite(M->de[s]) || !isfinite(M->e_lo[s]) || M->e_lo[s] < 0)
            return set_arg_error("lsm_model_create: energy bins must have de > 0, e_lo >= 0");
    if (!M->w || !M->mix_c || !M->mix_mu || !M->mix_sa || !M->mix_sb || !M->e_sa || !M->e_sb)
        return set_arg_error("lsm_model_create: NULL model array");
    const int ne = M->n_e, nr = M->n_r;
    const size_t nw = 3 * (size_t)ne * nr, nm = (size_t)ne * nr * 3, nes = (size_t)ne * nr;
    if (!finite_nonneg(M->w, nw)) return set_arg_error("lsm_model_create: PSR weights must be finite, >= 0");
    if (!finite_nonneg(M->mix_c, nm)) return set_arg_error("lsm_model_create: mixture weights must be >= 0");
    for (size_t i = 0; i < nes; ++i) {
        const double *c = M->mix_c + 3 * i;
        if (!(c[0] + c[1] + c[2] > 0)) return set_arg_error("lsm_model_create: mixture weights sum to 0");
        for (int k = 0; k < 3; ++k) {
            const double mu = M->mix_mu[3 * i + k], sa = M->mix_sa[3 * i + k], sb = M->mix_sb[3 * i + k];
            if (!(sa >= 0) || !(sb >= 0) || !(fabs(mu) + 5.8 * sa < 0.5 * kPiD) || !(5.8 * sb < 0.5 * kPiD))
                return set_arg_error("lsm_model_create: scatter direction mixture out of range");
        }
        if (!(M->e_sa[i] >= 0) || !(M->e_sb[i] >= 0) || !(5.8 * M->e_sa[i] < 0.5 * kPiD) ||
            !(5.8 * M->e_sb[i] < 0.5 * kPiD))
            return set_arg_error("lsm_model_create: electron direction widths out of range");
    }
    return LSM_OK;
}

lsm_status model_create(const lsm_psr_model *M, lsm_model **out)
{
    if (!M || !out) return set_arg_error("lsm_model_create: NULL argument");
    *out = nullptr;
    if (lsm_status rc = validate_model(M)) return rc;
    const size_t nw = 3 * (size_t)M->n_e * M->n_r, nm = (size_t)M->n_e * M->n_r * 3, nes = (size_t)M->n_e * M->n_r;
    lsm_model *h = (lsm_model *)calloc(1, sizeof(lsm_model));
    double *d = (double *)malloc((nw + 4 * nm + 2 * nes) * sizeof(double));
    if (!h || !d) { free(h); free(d); return set_arg_error("lsm_model_create: out of host memory"); }
    h->m = *M;
    h->data = d;
    auto put = [&](const double *src, size_t n) { memcpy(d, src, n * sizeof(double)); const double *p = d; d += n; return p; };
    h->m.w = put(M->w, nw);
    h->m.mix_c = put(M->mix_c, nm);
    h->m.mix_mu = put(M->mix_mu, nm);
    h->m.mix_sa = put(M->mix_sa, nm);
    h->m.mix_sb = put(M->mix_sb, nm);
    h->m.e_sa = put(M->e_sa, nes);
    h->m.e_sb = put(M->e_sb, nes);
    *out = h;
    return LSM_OK;
}

void model_destroy(lsm_model *h)
{
    if (!h) return;
    free(h->data);
    free(h);
}

lsm_status model_weights(const lsm_model *h, double *w)
{
    if (!h || !w) return set_arg_error("lsm_model_weights: NULL argument");
    memcpy(w, h->m.w, (size_t)3 * h->m.n_e * h->m.n_r * sizeof(double));
    return LSM_OK;
}

// The commissioned model (Sec. 2.2.4): PSR weights W_R scaled by the fitted
// factors x, either one per PSR (3 n_e n_r) or one per unknown of Eq. 8
// (2 n_e n_r photon PSRs, then one per electron energy bin applied to every
// ring of that bin).
lsm_status model_commission(const lsm_model *h, const double *x, int32_t n_x, lsm_model **out)
{
    if (!h || !x || !out) return set_arg_error("lsm_model_commission: NULL argument");
    *out = nullptr;
    const int ne = h->m.n_e, nr = h->m.n_r, n_ph = 2 * ne * nr;
    if (n_x != 3 * ne * nr && n_x != n_ph + ne)
        return set_arg_error("lsm_model_commission: x needs 3 n_e n_r (per PSR) or 2 n_e n_r + n_e (per unit) values");
    for (int i = 0; i < n_x; ++i)
        if (!(x[i] >= 0) || !isfinite(x[i])) return set_arg_error("lsm_model_commission: x must be finite, >= 0");
    std::vector<double> w((size_t)3 * ne * nr);
    for (int k = 0; k < 3 * ne * nr; ++k) {
        const double f = n_x == 3 * ne * nr ? x[k] : (k < n_ph ? x[k] : x[n_ph + (k - n_ph) / nr]);
        w[k] = h->m.w[k] * f;
    }
    lsm_psr_model m = h->m;
    m.w = w.data();
    return model_create(&m, out);
}

lsm_status build_psl(const lsm_model *Mh, const lsm_beams *B, int64_t n_hist,
                     const int64_t *per_psr_hist, lsm_psl **out, cudaStream_t st, bool async)
{
    if (!Mh || !B || !out) return set_arg_error("lsm_build_psl: NULL argument");
    *out = nullptr;
    const lsm_psr_model *M = &Mh->m;     // validated by lsm_model_create
    const int ne = M->n_e, nr = M->n_r, nxy = 2 * nr, npsl = nxy * nxy;
    const size_t nw = 3 * (size_t)ne * nr, nm = (size_t)ne * nr * 3, nes = (size_t)ne * nr;
    if (B->n_beams < 1 || B->n_beams > 16 || !B->jaws) return set_arg_error("lsm_build_psl: 1..16 beams");
    if (!(B->sad > B->z_jaw_x && B->z_jaw_x > M->z_phsp && B->sad > B->z_jaw_y && B->z_jaw_y > M->z_phsp))
        return set_arg_error("lsm_build_psl: need z_phsp < jaw planes < sad");
    for (int b = 0; b < B->n_beams; ++b) {
        const double *j = B->jaws + 4 * b;
        if (!(j[0] < j[1]) || !(j[2] < j[3]) || !isfinite(j[0]) || !isfinite(j[1]) || !isfinite(j[2]) ||
            !isfinite(j[3]))
            return set_arg_error("lsm_build_psl: jaws need x1 < x2 and y1 < y2");
        if (B->gantry && !(fabs(B->gantry[b]) <= 4.0 * kPiD))
            return set_arg_error("lsm_build_psl: gantry angles must be finite, |angle| <= 4 pi");
    }
    if (B->gantry && !(isfinite(B->iso[0]) && isfinite(B->iso[1]) && isfinite(B->iso[2])))
        return set_arg_error("lsm_build_psl: isocentre must be finite");
    const int nb = B->n_beams;
    const int npsr = 3 * ne * nr;
    if (!per_psr_hist && n_hist < 1) return set_arg_error("lsm_build_psl: n_hist must be >= 1");
    if (per_psr_hist)
        for (int k = 0; k < npsr; ++k)
            if (per_psr_hist[k] < 0) return set_arg_error("lsm_build_psl: negative per-PSR history count");

    lsm_psl *P = (lsm_psl *)calloc(1, sizeof(lsm_psl));
    if (!P) return set_arg_error("lsm_build_psl: out of host memory");
    P->uid = next_uid();
    cudaGetDevice(&P->device);
    P->n_e = ne; P->n_r = nr; P->n_xy = nxy; P->n_beams = nb; P->per_psr = per_psr_hist != nullptr;
    P->dr = M->dr; P->z_phsp = M->z_phsp; P->sigma_s = M->sigma_s;
    for (int s = 0; s < 3; ++s) { P->e_lo[s] = M->e_lo[s]; P->de[s] = M->de[s]; }
    P->sad = B->sad; P->z_jaw_y = B->z_jaw_y; P->z_jaw_x = B->z_jaw_x;
    P->rotated = B->gantry != nullptr;
    for (int b = 0; b < nb; ++b) P->gantry[b] = B->gantry ? B->gantry[b] : 0.0;
    for (int k = 0; k < 3; ++k) P->iso[k] = B->gantry ? B->iso[k] : (k == 2 ? B->sad : 0.0);
    const int64_t ncell = P->per_psr ? (int64_t)npsr * nb * npsl : (int64_t)nb * 3 * ne * npsl;
    P->ncell = ncell;

    // One device allocation holds every table of the plan and the scratch of
    // the build (released only by lsm_psl_destroy). It is stream-ordered
    // (cudaMallocAsync from the device's memory pool): a build neither waits
    // for the device nor makes the device wait for it.
    const size_t nbse = (size_t)nb * 3 * ne;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_in = take((nw + 4 * nm + 2 * nes + 4 * (size_t)nb + (size_t)npsr) * 8);
    const size_t o_wpsl = take(3 * (size_t)ne * npsl * 8), o_scale = take(3 * (size_t)ne * 8);
    const size_t o_jf = take((size_t)nb * 16), o_area = take((size_t)nb * 64), o_incl = take((size_t)nb * 2 * npsl);
    const size_t o_count = take((size_t)ncell * 8), o_r0 = take((size_t)npsl * 4), o_l0 = take((size_t)npsl * 8);
    const size_t o_thr = take(nes * 16), o_mix = take(nes * 3 * sizeof(float4)), o_esig = take(nes * sizeof(float2));
    const size_t o_start = take((size_t)(ncell + 1) * 8), o_ent = take((size_t)ncell * sizeof(EntryRec));
    const size_t o_esc = take((size_t)ncell * 8);
    const size_t o_rem = take((size_t)ncell * 8), o_cst = take((size_t)(ncell + 1) * 8);
    const size_t o_eidx = take((size_t)(ncell + 1) * 8), o_parts = take(nbse * 8);
    const size_t o_res = take(64), o_dkb = take((size_t)npsr * nb * 8);
    const size_t o_rot = take((size_t)nb * sizeof(float2));
    char *base = nullptr;
    {
        cudaError_t e_ = cudaMallocAsync((void **)&base, off, st);
        if (e_ != cudaSuccess) { free_psl(P); return set_cuda_error(e_, "lsm_build_psl: cudaMallocAsync"); }
    }
    P->arena = base;
    double *d_in = (double *)(base + o_in);
    P->d_w = d_in;
    double *d_mc = d_in + nw, *d_mmu = d_mc + nm, *d_msa = d_mmu + nm, *d_msb = d_msa + nm;
    double *d_esa = d_msb + nm, *d_esb = d_esa + nes;
    P->d_jaws = d_esb + nes;
    int64_t *d_nk = (int64_t *)(P->d_jaws + 4 * nb);
    P->d_wpsl = (double *)(base + o_wpsl); P->d_scale = (double *)(base + o_scale);
    P->d_jaws_f = (float *)(base + o_jf); P->d_area = (double *)(base + o_area); P->d_incl = (uint8_t *)(base + o_incl);
    P->d_count = (int64_t *)(base + o_count); P->d_tag_r0 = (int32_t *)(base + o_r0); P->d_tag_l0 = (double *)(base + o_l0);
    P->d_mixthr = (unsigned long long *)(base + o_thr); P->d_mix = (float4 *)(base + o_mix);
    P->d_esig = (float2 *)(base + o_esig);
    P->d_start = (int64_t *)(base + o_start); P->d_ent = (EntryRec *)(base + o_ent); P->d_escale = (double *)(base + o_esc);
    double *d_rem = (double *)(base + o_rem);
    int64_t *d_cstart = (int64_t *)(base + o_cst), *d_eidx = (int64_t *)(base + o_eidx);
    double *d_parts = (double *)(base + o_parts);
    double *d_denom = (double *)(base + o_res);
    unsigned long long *d_fsum = (unsigned long long *)(base + o_res + 8);
    double *d_dkb = (double *)(base + o_dkb);

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) { free_psl(P); return set_cuda_error(e_, #call); } \
    } while (0)
#define CKL(where)                                               \
    do {                                                         \
        count_launch();                                          \
        cudaError_t e_ = cudaGetLastError();                     \
        if (e_ != cudaSuccess) { free_psl(P); return set_cuda_error(e_, where); } \
    } while (0)

    // host inputs packed into one copy from pinned memory (a copy from
    // pageable memory would first wait for the stream's earlier work). Each
    // thread keeps a ring of four staging buffers, each with an event recorded
    // after the copies out of it: a buffer is refilled only once its copies
    // have run, so that builds queued without host synchronisation behind
    // other work never overwrite inputs still waiting to be copied.
    const size_t n_in = nw + 4 * nm + 2 * nes + 4 * (size_t)nb + (size_t)npsr;
    struct Stage {
        double *buf;
        size_t cap;
        cudaEvent_t copied;
    };
    static thread_local Stage ring[4] = {};
    static thread_local int ring_next = 0;
    Stage &sg = ring[ring_next];
    ring_next = (ring_next + 1) & 3;
    if (sg.copied) CK(cudaEventSynchronize(sg.copied));
    if (!sg.copied) CK(cudaEventCreateWithFlags(&sg.copied, cudaEventDisableTiming));
    if (sg.cap < n_in + 24) {
        if (sg.buf) cudaFreeHost(sg.buf);
        sg.buf = nullptr;
        sg.cap = 0;
        CK(cudaMallocHost((void **)&sg.buf, (n_in + 24) * sizeof(double)));
        sg.cap = n_in + 24;
    }
    double *const hbuf = sg.buf;
    {
        double *h = hbuf;
        memset(h, 0, n_in * sizeof(double));
        memcpy(h, M->w, nw * 8); h += nw;
        memcpy(h, M->mix_c, nm * 8); h += nm;
        memcpy(h, M->mix_mu, nm * 8); h += nm;
        memcpy(h, M->mix_sa, nm * 8); h += nm;
        memcpy(h, M->mix_sb, nm * 8); h += nm;
        memcpy(h, M->e_sa, nes * 8); h += nes;
        memcpy(h, M->e_sb, nes * 8); h += nes;
        memcpy(h, B->jaws, (size_t)nb * 32); h += 4 * nb;
        if (per_psr_hist) memcpy(h, per_psr_hist, (size_t)npsr * 8);
    }
    CK(cudaMemcpyAsync(d_in, hbuf, n_in * 8, cudaMemcpyHostToDevice, st));
    {
        float2 *hrot = (float2 *)(hbuf + n_in);       // 16 beams x 8 bytes in the 16 spare slots
        for (int b = 0; b < nb; ++b) hrot[b] = make_float2((float)cos(P->gantry[b]), (float)sin(P->gantry[b]));
        CK(cudaMemcpyAsync(base + o_rot, hrot, (size_t)nb * sizeof(float2), cudaMemcpyHostToDevice, st));
    }
    CK(cudaEventRecord(sg.copied, st));
    CK(cudaMemsetAsync(d_denom, 0, 64, st));

    {
        SetupArgs A;
        A.w = P->d_w; A.n_e = ne; A.n_r = nr; A.dr = M->dr;
        A.wpsl = P->d_wpsl; A.block_scale = P->d_scale; A.tag_r0 = P->d_tag_r0; A.tag_l0 = P->d_tag_l0;
        A.G.jaws = P->d_jaws; A.G.n_beams = nb; A.G.z_phsp = M->z_phsp; A.G.sad = B->sad;
        A.G.z_jaw_x = B->z_jaw_x; A.G.z_jaw_y = B->z_jaw_y;
        A.area = P->d_area; A.jaws_f = P->d_jaws_f; A.incl = P->d_incl;
        A.n_incl_blocks = (int)(((int64_t)nb * 2 * npsl + 255) / 256);
        A.mc = d_mc; A.mmu = d_mmu; A.msa = d_msa; A.msb = d_msb; A.esa = d_esa; A.esb = d_esb;
        A.nes = (int)nes; A.thr = P->d_mixthr; A.mix = P->d_mix; A.esig = P->d_esig;
        const unsigned grid = (unsigned)(3 * ne + A.n_incl_blocks + (int)((nes + 255) / 256));
        if ((size_t)npsl * 8 > 48 * 1024)
            CK(cudaFuncSetAttribute(k_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, npsl * 8));
        k_setup<<<grid, 256, (size_t)npsl * 8, st>>>(A);
        CKL("k_setup");
    }

    if (!per_psr_hist) {
        const int nb3 = (int)nbse;
        if ((size_t)npsl * 8 > 48 * 1024)
            CK(cudaFuncSetAttribute(k_eq3_parts, cudaFuncAttributeMaxDynamicSharedMemorySize, npsl * 8));
        k_eq3_parts<<<nb3, 256, (size_t)npsl * 8, st>>>(P->d_wpsl, P->d_incl, nb, ne, npsl, d_parts);
        CKL("k_eq3_parts");
        const unsigned g = (unsigned)((ncell + 255) / 256);
        k_eq3_floor<<<g, 256, 0, st>>>(P->d_wpsl, P->d_incl, ne, npsl, ncell, n_hist, d_parts, nb3, d_denom,
                                       P->d_count, d_rem, d_fsum);
        CKL("k_eq3_floor");
        k_eq3_select<<<1, 1024, 0, st>>>(d_rem, ncell, n_hist, d_fsum, d_denom, P->d_count, d_cstart, d_eidx,
                                         P->d_start, (int64_t *)(base + o_res + 16));
        CKL("k_eq3_select");
    } else {
        const size_t smem = (size_t)npsl * 24;
        if (smem > 48 * 1024) CK(cudaFuncSetAttribute(k_psr_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_psr_counts<<<npsr * nb, 256, smem, st>>>(P->d_w, P->d_scale, P->d_incl, d_nk, ne, nr, M->dr, nb,
                                                   P->d_count, d_dkb);
        CKL("k_psr_counts");
    }
    if (per_psr_hist) {      // (the whole-source plan's scans ran in k_eq3_select)
        k_scan_counts<<<1, 1024, 0, st>>>(P->d_count, ncell, d_cstart, d_eidx, P->d_start,
                                          (int64_t *)(base + o_res + 16));
        CKL("k_scan_counts");
    }
    k_entries<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(P->d_count, d_cstart, d_eidx, ncell, P->per_psr, nb, ne,
                                                              nr, P->d_w, P->d_tag_r0, P->d_tag_l0, d_dkb, d_nk,
                                                              P->d_start, P->d_ent, P->d_escale);
    CKL("k_entries");
    // (denominator, floor sum, n_ent, total) are contiguous: one copy into the
    // plan's pinned slot, then the plan's completion event
    P->h_res = take_slot();
    if (!P->h_res) { free_psl(P); return set_arg_error("lsm_build_psl: out of pinned host memory"); }
    {
        cudaEvent_t ev = nullptr;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        P->done = ev;
    }
    CK(cudaMemcpyAsync(P->h_res, base + o_res, 32, cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord((cudaEvent_t)P->done, st));
    P->denom = 0.0;
    P->n_ent = -1;
    // a whole-source plan distributes exactly n_hist histories unless its
    // areas are empty (reported when the results are read)
    P->plan_size = per_psr_hist ? -1 : n_hist;
    if (!async || per_psr_hist) {
        const lsm_status r = resolve_psl(P);
        if (r) { free_psl(P); return r; }
    }

    SampleParams &sp = P->sp;
    sp.start = P->d_start; sp.ent = P->d_ent; sp.mixthr = P->d_mixthr; sp.mix = P->d_mix; sp.esig = P->d_esig;
    sp.jaws_f = P->d_jaws_f; sp.n_ent = (const int64_t *)(base + o_res + 16); sp.n_e = ne; sp.n_r = nr;
    sp.pitch = (float)M->dr; sp.z_phsp = (float)M->z_phsp; sp.sigma_s = (float)M->sigma_s;
    for (int s = 0; s < 3; ++s) { sp.e_lo[s] = (float)M->e_lo[s]; sp.de[s] = (float)M->de[s]; }
    sp.zy_rel = (float)(B->z_jaw_y - M->z_phsp);
    sp.zx_rel = (float)(B->z_jaw_x - M->z_phsp);
    sp.rot = (const float2 *)(base + o_rot);
    for (int k = 0; k < 3; ++k) sp.iso[k] = (float)P->iso[k];
    sp.sad = (float)B->sad;
    sp.rotated = P->rotated;
    *out = P;
    return LSM_OK;
#undef CK
#undef CKL
}

// The arena returns to the pool in the order of the legacy default stream,
// i.e. after the work already queued on the blocking streams; work that uses
// the plan on other streams must be complete (lsm_psl_destroy's contract).
lsm_status free_psl(lsm_psl *P)
{
    if (!P) return LSM_OK;
    if (P->done) {
        // the result copy must have landed before the slot is reused
        cudaEventSynchronize((cudaEvent_t)P->done);
        cudaEventDestroy((cudaEvent_t)P->done);
    }
    give_slot(P->h_res);
    if (P->arena) cudaFreeAsync(P->arena, 0);
    free(P);
    return LSM_OK;
}

}  // namespace lsm
