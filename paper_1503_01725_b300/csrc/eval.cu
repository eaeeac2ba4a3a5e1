// eval.cu -- judging a dose estimate against a reference dose on the GPU:
// the global gamma index (Low, Harms, Mutic & Purdy 1998) and the RMS
// relative error over the high-dose region with the reference's own variance
// removed.
//
// Gamma: for each reference voxel above threshold * Dmax_ref, the minimum over
// points r of |r - r_ref|^2 / DTA^2 + (D_eval(r) - D_ref)^2 / (c Dmax_ref)^2
// is compared with 1. Only points within DTA can pass, so the search runs over
// the DTA sphere on a grid of step `step_mm`, nearest offsets first, stopping
// at the first that passes; D_eval is interpolated trilinearly with the edge
// value continued outside the volume.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace lsm {
namespace {

__global__ void k_fmax(const float *__restrict__ a, long long n, unsigned *out_bits)
{
    unsigned m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fmaxf(a[i], 0.0f)));
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, m);
}

__device__ __forceinline__ float trilinear(const float *__restrict__ v, int d, int h, int w, float z, float y, float x)
{
    z = fminf(fmaxf(z, 0.0f), (float)(d - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    const int z0 = min((int)z, d - 1), y0 = min((int)y, h - 1), x0 = min((int)x, w - 1);
    const int z1 = min(z0 + 1, d - 1), y1 = min(y0 + 1, h - 1), x1 = min(x0 + 1, w - 1);
    const float fz = z - z0, fy = y - y0, fx = x - x0;
    auto at = [&](int a, int b, int c) { return v[((long long)a * h + b) * w + c]; };
    const float c00 = at(z0, y0, x0) + fx * (at(z0, y0, x1) - at(z0, y0, x0));
    const float c01 = at(z0, y1, x0) + fx * (at(z0, y1, x1) - at(z0, y1, x0));
    const float c10 = at(z1, y0, x0) + fx * (at(z1, y0, x1) - at(z1, y0, x0));
    const float c11 = at(z1, y1, x0) + fx * (at(z1, y1, x1) - at(z1, y1, x0));
    const float c0 = c00 + fy * (c01 - c00), c1 = c10 + fy * (c11 - c10);
    return c0 + fz * (c1 - c0);
}

// offs[k] = (dz, dy, dx in voxel units, squared distance / DTA^2), nearest first
__global__ void k_gamma(const float *__restrict__ ev, const float *__restrict__ ref, int d, int h, int w,
                        const float4 *__restrict__ offs, int n_offs, const unsigned *__restrict__ dmax_bits,
                        float dose_crit, float threshold, unsigned long long *counts, unsigned char *pass_map)
{
    const float dmax = __uint_as_float(*dmax_bits);
    const float inv_crit = 1.0f / (dose_crit * dmax);
    const long long n = (long long)d * h * w;
    unsigned long long roi = 0, ok = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float r = ref[i];
        unsigned char flag = 0;
        if (r > threshold * dmax) {
            ++roi;
            const int x = (int)(i % w), y = (int)((i / w) % h), z = (int)(i / ((long long)w * h));
            for (int k = 0; k < n_offs; ++k) {
                const float4 o = offs[k];
                const float de = trilinear(ev, d, h, w, z + o.x, y + o.y, x + o.z);
                const float t = (de - r) * inv_crit;
                if (o.w + t * t <= 1.0f) {
                    flag = 1;
                    break;
                }
            }
            ok += flag;
            flag |= 2;
        }
        if (pass_map) pass_map[i] = flag;
    }
    for (int s = 16; s; s >>= 1) {
        roi += __shfl_xor_sync(0xFFFFFFFFu, roi, s);
        ok += __shfl_xor_sync(0xFFFFFFFFu, ok, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts, roi);
        atomicAdd(counts + 1, ok);
    }
}

// sums over voxels with ref > level * Dmax: ((est - ref) / ref)^2, (sigma / ref)^2, count
__global__ void k_dose_err(const float *__restrict__ est, const float *__restrict__ ref, const float *__restrict__ sig,
                           long long n, const unsigned *__restrict__ dmax_bits, float level, double *sums)
{
    const float thr = level * __uint_as_float(*dmax_bits);
    double e = 0.0, s = 0.0, c = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float r = ref[i];
        if (r > thr) {
            const double q = ((double)est[i] - r) / r;
            e += q * q;
            if (sig) {
                const double t = (double)sig[i] / r;
                s += t * t;
            }
            c += 1.0;
        }
    }
    for (int o = 16; o; o >>= 1) {
        e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
        s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, e);
        atomicAdd(sums + 1, s);
        atomicAdd(sums + 2, c);
    }
}

int grid_for_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 16ll * sm_count())); }

// device copies of host arrays when mem is HOST; released by the caller
// Curve comparison (Eq. 10-11 and distance to agreement, Sec. 3.2) in one
// CTA: each thread takes measured points, searches every segment of the
// piecewise-linear calculated curve for the measured value, and the CTA
// reduces sum of squares, max |difference|, DTA sum / max and counts.
__global__ void k_curve(const float *__restrict__ pos, const float *__restrict__ calc, const float *__restrict__ meas,
                        int n, double lo, double hi, int use_abs, double *out)
{
    double ss = 0.0, mx = 0.0, dsum = 0.0, dmax = 0.0;
    int cnt = 0, nocross = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = pos[i], key = use_abs ? fabs(x) : x;
        if (!(key >= lo && key < hi)) continue;
        const double m = meas[i], d = (double)calc[i] - m;
        ss += d * d;
        mx = fmax(mx, fabs(d));
        ++cnt;
        double best = INFINITY;
        for (int j = 0; j + 1 < n; ++j) {
            const double c0 = calc[j], c1 = calc[j + 1], y0 = pos[j], y1 = pos[j + 1];
            double dist;
            if (c0 == c1) {
                if (c0 != m) continue;
                dist = (y0 <= x && x <= y1) ? 0.0 : fmin(fabs(x - y0), fabs(x - y1));
            } else {
                // the end segments continue beyond the first and last points
                const double t = (m - c0) / (c1 - c0);
                if (!((t >= 0.0 && t <= 1.0) || (j == 0 && t < 0.0) || (j == n - 2 && t > 1.0))) continue;
                dist = fabs(x - (y0 + t * (y1 - y0)));
            }
            best = fmin(best, dist);
        }
        if (isinf(best)) ++nocross;
        else { dsum += best; dmax = fmax(dmax, best); }
    }
    __shared__ double sh[4][256];
    __shared__ int shc[2][256];
    sh[0][threadIdx.x] = ss; sh[1][threadIdx.x] = mx; sh[2][threadIdx.x] = dsum; sh[3][threadIdx.x] = dmax;
    shc[0][threadIdx.x] = cnt; shc[1][threadIdx.x] = nocross;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
            sh[2][threadIdx.x] += sh[2][threadIdx.x + o];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + o]);
            shc[0][threadIdx.x] += shc[0][threadIdx.x + o];
            shc[1][threadIdx.x] += shc[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0]; out[1] = sh[1][0]; out[2] = sh[2][0]; out[3] = sh[3][0];
        out[4] = shc[0][0]; out[5] = shc[1][0];
    }
}

struct Staged {
    std::vector<void *> bufs;
    ~Staged()
    {
        for (void *p : bufs) cudaFree(p);
    }
    const float *put(const float *src, long long n, lsm_mem mem, cudaStream_t st, cudaError_t &e)
    {
        if (!src || mem == LSM_MEM_DEVICE || e != cudaSuccess) return src;
        void *p = nullptr;
        if ((e = cudaMalloc(&p, (size_t)n * 4)) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        e = cudaMemcpyAsync(p, src, (size_t)n * 4, cudaMemcpyHostToDevice, st);
        return (const float *)p;
    }
};

// FP32 atomic adds, result unused, at pseudo-random cells: thread i walks the
// LCG x -> 1664525 x + 1013904223 (mod 2^32; Numerical Recipes, Sec. 7.1) from
// x = i and maps each state to a cell by a 32x32 -> high-32 multiply, as the
// transport's tally updates land on scattered voxels
__global__ void k_atomic_peak(float *__restrict__ cells, uint32_t n_cells, int per_thread)
{
    uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < per_thread; ++i) {
        x = x * 1664525u + 1013904223u;
        atomicAdd(cells + __umulhi(x, n_cells), 1.0f);
    }
}

// Philox4x32-10 blocks of the transport's streams: block i at counter
// (g lo, g hi, stream id, draw) for history g = g0 + i
// (four 32-bit stores: the caller's array needs only 4-byte alignment)
__global__ void k_philox(uint32_t k0, uint32_t k1, uint64_t g0, uint32_t sid, uint32_t draw, int64_t n,
                         uint32_t *__restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t g = g0 + (uint64_t)i;
        const uint4 r = philox4x32_10(k0, k1, (uint32_t)g, (uint32_t)(g >> 32), sid, draw);
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

}  // namespace
}  // namespace lsm

using namespace lsm;

extern "C" {

lsm_status lsm_gamma(const float *eval, const float *ref, int32_t d, int32_t h, int32_t w, const double voxel_mm[3],
                     double dose_crit, double dta_mm, double threshold, double step_mm, lsm_mem mem,
                     double *pass_rate, int64_t *n_roi, unsigned char *pass_map, lsm_stream stream)
{
    if (!eval || !ref || !voxel_mm || !pass_rate) return set_arg_error("lsm_gamma: NULL argument");
    if (d < 1 || h < 1 || w < 1 || dose_crit <= 0 || dta_mm <= 0 || step_mm <= 0 || threshold < 0 ||
        voxel_mm[0] <= 0 || voxel_mm[1] <= 0 || voxel_mm[2] <= 0 || dta_mm / step_mm > 40)
        return set_arg_error("lsm_gamma: sizes, criteria and step must be positive (DTA / step <= 40)");
    const cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)d * h * w;
    // search offsets in the DTA sphere, nearest first
    const int k = (int)floor(dta_mm / step_mm + 1e-9);
    std::vector<float4> offs;
    std::vector<double> r2s;
    for (int a = -k; a <= k; ++a)
        for (int b = -k; b <= k; ++b)
            for (int c = -k; c <= k; ++c) {
                const double oz = a * step_mm, oy = b * step_mm, ox = c * step_mm;
                const double r2 = oz * oz + oy * oy + ox * ox;
                if (r2 > dta_mm * dta_mm + 1e-12) continue;
                offs.push_back(make_float4((float)(oz / voxel_mm[0]), (float)(oy / voxel_mm[1]),
                                           (float)(ox / voxel_mm[2]), (float)(r2 / (dta_mm * dta_mm))));
                r2s.push_back(r2);
            }
    std::vector<int> ord(offs.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return r2s[x] < r2s[y]; });
    std::vector<float4> sorted(offs.size());
    for (size_t i = 0; i < ord.size(); ++i) sorted[i] = offs[ord[i]];
    cudaError_t e = cudaSuccess;
    Staged S;
    const float *dev = S.put(eval, n, mem, st, e);
    const float *dref = S.put(ref, n, mem, st, e);
    void *work = nullptr;
    unsigned char *dmap = nullptr;
    const size_t wbytes = 256 + sorted.size() * sizeof(float4);
    if (e == cudaSuccess) e = cudaMalloc(&work, wbytes);
    if (e == cudaSuccess && pass_map) e = cudaMalloc(&dmap, (size_t)n);
    if (e != cudaSuccess) {
        cudaFree(work);
        cudaFree(dmap);
        return set_cuda_error(e, "lsm_gamma");
    }
    unsigned long long *counts = (unsigned long long *)work;
    unsigned *dmax = (unsigned *)((char *)work + 64);
    float4 *doffs = (float4 *)((char *)work + 256);
    unsigned long long host_counts[2] = {0, 0};
    do {
        if ((e = cudaMemsetAsync(work, 0, 256, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(doffs, sorted.data(), sorted.size() * sizeof(float4), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            break;
        k_fmax<<<grid_for_n(n), 256, 0, st>>>(dref, n, dmax);
        count_launch();
        k_gamma<<<grid_for_n(n), 256, 0, st>>>(dev, dref, d, h, w, doffs, (int)sorted.size(), dmax, (float)dose_crit,
                                               (float)threshold, counts, dmap);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(host_counts, counts, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if (pass_map &&
            (e = cudaMemcpyAsync(pass_map, dmap, (size_t)n,
                                 mem == LSM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess)
            break;
        e = cudaStreamSynchronize(st);
    } while (0);
    cudaFree(work);
    cudaFree(dmap);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_gamma");
    *pass_rate = host_counts[0] ? (double)host_counts[1] / (double)host_counts[0] : 1.0;
    if (n_roi) *n_roi = (int64_t)host_counts[0];
    return LSM_OK;
}

lsm_status lsm_dose_error(const float *est, const float *ref, const float *sigma_ref, int64_t n, double level,
                          lsm_mem mem, double *rms_rel, lsm_stream stream)
{
    if (!est || !ref || !rms_rel) return set_arg_error("lsm_dose_error: NULL argument");
    if (n < 1 || level < 0) return set_arg_error("lsm_dose_error: n >= 1, level >= 0");
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    Staged S;
    const float *de = S.put(est, n, mem, st, e);
    const float *dr = S.put(ref, n, mem, st, e);
    const float *ds = S.put(sigma_ref, n, mem, st, e);
    void *work = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&work, 128);
    double sums[3] = {0, 0, 0};
    do {
        if (e != cudaSuccess) break;
        if ((e = cudaMemsetAsync(work, 0, 128, st)) != cudaSuccess) break;
        unsigned *dmax = (unsigned *)((char *)work + 64);
        k_fmax<<<grid_for_n(n), 256, 0, st>>>(dr, n, dmax);
        count_launch();
        k_dose_err<<<grid_for_n(n), 256, 0, st>>>(de, dr, ds, n, dmax, (float)level, (double *)work);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(sums, work, 24, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        e = cudaStreamSynchronize(st);
    } while (0);
    cudaFree(work);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_dose_error");
    const double cnt = sums[2] > 0 ? sums[2] : 1.0;
    *rms_rel = sqrt(std::max(sums[0] / cnt - sums[1] / cnt, 0.0));
    return LSM_OK;
}

lsm_status lsm_curve_compare(const float *pos, const float *calc, const float *meas, int32_t n, double lo, double hi,
                             int32_t use_abs, double dmax_m, lsm_mem mem, double out[6], lsm_stream stream)
{
    if (!pos || !calc || !meas || !out) return set_arg_error("lsm_curve_compare: NULL argument");
    if (n < 2 || n > (1 << 20) || !(dmax_m > 0)) return set_arg_error("lsm_curve_compare: 2 <= n <= 2^20, dmax_m > 0");
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    Staged S;
    const float *dp = S.put(pos, n, mem, st, e);
    const float *dc = S.put(calc, n, mem, st, e);
    const float *dm = S.put(meas, n, mem, st, e);
    double *work = nullptr, r[6] = {0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMalloc(&work, 6 * sizeof(double));
    if (e == cudaSuccess) {
        k_curve<<<1, 256, 0, st>>>(dp, dc, dm, n, lo, hi, use_abs, work);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, work, sizeof(r), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(work);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_curve_compare");
    const double cnt = r[4], fin = r[4] - r[5];
    out[0] = cnt > 0 ? sqrt(r[0] / cnt) / dmax_m : 0.0;
    out[1] = r[1] / dmax_m;
    out[2] = fin > 0 ? r[2] / fin : 0.0;
    out[3] = r[3];
    out[4] = r[4];
    out[5] = r[5];
    return LSM_OK;
}

lsm_status lsm_l2_atomic_peak(int64_t n_cells, int32_t reps, double *atomics_per_s, lsm_stream stream)
{
    if (!atomics_per_s) return set_arg_error("lsm_l2_atomic_peak: NULL argument");
    if (n_cells < 1 || n_cells > (1ll << 31) || reps < 1 || reps > 1000)
        return set_arg_error("lsm_l2_atomic_peak: 1 <= n_cells <= 2^31, 1 <= reps <= 1000");
    const cudaStream_t st = (cudaStream_t)stream;
    constexpr int kThreads = 256, kPer = 256;
    const int grid = 8 * sm_count();
    const double per_launch = (double)grid * kThreads * kPer;
    float *cells = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    cudaError_t e = dev_malloc((void **)&cells, (size_t)n_cells * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cells, 0, (size_t)n_cells * 4, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {   // warm-up
        k_atomic_peak<<<grid, kThreads, 0, st>>>(cells, (uint32_t)n_cells, kPer);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        k_atomic_peak<<<grid, kThreads, 0, st>>>(cells, (uint32_t)n_cells, kPer);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cells) dev_free(cells);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_l2_atomic_peak");
    *atomics_per_s = ms > 0.0f ? per_launch * reps / (ms * 1e-3) : 0.0;
    return LSM_OK;
}

lsm_status lsm_philox_blocks(uint64_t seed, uint64_t first_history, uint32_t stream_id, uint32_t draw, int64_t n,
                             uint32_t *out, lsm_mem mem, lsm_stream stream)
{
    if (!out) return set_arg_error("lsm_philox_blocks: NULL argument");
    if (n < 1 || n > (1ll << 28)) return set_arg_error("lsm_philox_blocks: 1 <= n <= 2^28");
    const cudaStream_t st = (cudaStream_t)stream;
    uint32_t *d = out;
    cudaError_t e = cudaSuccess;
    if (mem == LSM_MEM_HOST) e = dev_malloc((void **)&d, (size_t)n * 16, st);
    if (e == cudaSuccess) {
        k_philox<<<grid_for_n(n), 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), first_history, stream_id,
                                               draw, n, d);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && mem == LSM_MEM_HOST) {
        e = cudaMemcpyAsync(out, d, (size_t)n * 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (mem == LSM_MEM_HOST && d) dev_free(d);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_philox_blocks");
    return LSM_OK;
}

}  // extern "C"
