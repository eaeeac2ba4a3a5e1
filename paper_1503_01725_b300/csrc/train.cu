// train.cu -- training of the dose denoiser on the GPU.
//
// One step: the forward pass (denoise.cu, activations kept), the normalised
// MSE loss and its gradient through the 1x1x1 head, then for every conv layer
// in reverse order the ReLU mask of its output gradient, the bias gradient
// (a column sum), the weight gradient (FP32 CUDA-core reduction over voxels:
// dW[o][tap][c] = sum_v gz[v][o] x[v + tap][c]) and the data gradient (the
// tensor-core convolution of denoise.cu run with the weights mirrored in the
// three axes and transposed in channels); max-pool and upsampling backward and
// the sums of the skip branches; Adam on the FP32 master parameters; and the
// repacking of the updated weights into both operand images.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "unet.cuh"

namespace lsm {
namespace dn {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float bf(bf16 v) { return __bfloat162float(v); }

// ------------------------------------------------------------ weight packing ---
// Forward image of a (cin -> cout) layer with kc channels per stage (the
// layout the host packer of conv_create writes) and, when img_t is given, the
// image of the data-gradient layer (cout -> cin, kc_t per stage) whose weight
// is w[o][2-dz][2-dy][2-dx][c] at (c, dz, dy, dx, o).
__global__ void k_pack(const float *__restrict__ w, int cin, int cout, int kc, int kc_t, bf16 *__restrict__ img,
                       bf16 *__restrict__ img_t, const float *__restrict__ b, float *__restrict__ bias)
{
    const long long total = 27ll * cin * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % cin);
        long long r = i / cin;
        const int tap27 = (int)(r % 27);
        const int o = (int)(r / 27);
        const int dz = tap27 / 9, dy = (tap27 / 3) % 3, dx = tap27 % 3;
        const bf16 v = __float2bfloat16_rn(w[i]);
        img[wimg_offset(cout, kc, c / kc, dz, dy, dx, o, c % kc)] = v;
        // the data-gradient layer: input and output channels swapped, taps mirrored
        if (img_t) img_t[wimg_offset(cin, kc_t, o / kc_t, 2 - dz, 2 - dy, 2 - dx, c, o % kc_t)] = v;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cout; i += gridDim.x * blockDim.x)
        bias[i] = bf(__float2bfloat16_rn(b[i]));
}

// ------------------------------------------------------------- loss, head ---
// per voxel: r = hw . d0 + hb, res = dose / Dmax + r - target / Dmax;
// loss = mean res^2; g = 2 res / N; g_d0 = g hw (BF16); dhw += g d0; dhb += g
__global__ void k_head_train(const bf16 *__restrict__ d0, int ct, const float *__restrict__ hw,
                             const float *__restrict__ dose, const float *__restrict__ target,
                             const unsigned *__restrict__ dmax_bits, bf16 *__restrict__ g_d0, int g_ct,
                             float *__restrict__ g_head, double *__restrict__ loss, int n, VolIdx v, float inv_n)
{
    float acc[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) acc[c] = 0.0f;
    double l = 0.0;
    const long long per = (long long)v.d * v.h * v.w, total = per * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / per);
        long long r = i - (long long)b * per;
        const int xx = (int)(r % v.w); r /= v.w;
        const int yy = (int)(r % v.h);
        const int zz = (int)(r / v.h);
        const long long at = v.at(b, zz, yy, xx);
        float f[16];
        const uint4 *src = reinterpret_cast<const uint4 *>(d0 + at * ct);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint4 u = src[k];
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 p = __bfloat1622float2(h[j]);
                f[8 * k + 2 * j] = p.x;
                f[8 * k + 2 * j + 1] = p.y;
            }
        }
        float rr = hw[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) rr += hw[c] * f[c];
        const float dm = __uint_as_float(dmax_bits[b]);
        const float inv = dm > 0.0f ? 1.0f / dm : 0.0f;
        const float res = dose[i] * inv + rr - target[i] * inv;
        l += (double)res * res;
        const float g = 2.0f * res * inv_n;
        uint32_t pk[8];
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
            acc[c] += g * f[c];
            acc[c + 1] += g * f[c + 1];
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(g * hw[c], g * hw[c + 1]);
            pk[c / 2] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        acc[16] += g;
        uint4 *dst = reinterpret_cast<uint4 *>(g_d0 + at * g_ct);
        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
#pragma unroll
    for (int c = 0; c < 17; ++c)
        for (int o = 16; o; o >>= 1) acc[c] += __shfl_xor_sync(0xFFFFFFFFu, acc[c], o);
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 17; ++c) atomicAdd(g_head + c, acc[c]);
        atomicAdd(loss, l * (double)inv_n);
    }
}

// ----------------------------------------------------------- ReLU, bias ---
// gz = gy where the layer output y > 0, else 0 (interior voxels, 8-channel groups)
__global__ void k_relu_mask(const bf16 *__restrict__ gy, int gy_ct, int gy_co, const bf16 *__restrict__ y, int y_ct,
                            int y_co, bf16 *__restrict__ gz, int gz_ct, int groups, int n, VolIdx v)
{
    const long long total = (long long)n * v.d * v.h * v.w * groups;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % groups);
        long long r = i / groups;
        const int xx = (int)(r % v.w); r /= v.w;
        const int yy = (int)(r % v.h); r /= v.h;
        const int zz = (int)(r % v.d);
        const int b = (int)(r / v.d);
        const long long at = v.at(b, zz, yy, xx);
        uint4 gv = *reinterpret_cast<const uint4 *>(gy + at * gy_ct + gy_co + 8 * g);
        const uint4 yv = *reinterpret_cast<const uint4 *>(y + at * y_ct + y_co + 8 * g);
        const bf16 *ys = reinterpret_cast<const bf16 *>(&yv);
        bf16 *gs = reinterpret_cast<bf16 *>(&gv);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (!(bf(ys[k]) > 0.0f)) gs[k] = __float2bfloat16_rn(0.0f);
        *reinterpret_cast<uint4 *>(gz + at * gz_ct + 8 * g) = gv;
    }
}

// db[o] += sum over interior voxels of gz[v][o]
__global__ void k_bias_grad(const bf16 *__restrict__ gz, int ct, int c, int n, VolIdx v, float *__restrict__ db)
{
    __shared__ float red[256];
    const int rows = blockDim.x / c;
    const int ch = threadIdx.x % c, row = threadIdx.x / c;
    float s = 0.0f;
    const long long total = (long long)n * v.d * v.h * v.w;
    if (row < rows) {
        for (long long i = (long long)blockIdx.x * rows + row; i < total; i += (long long)gridDim.x * rows) {
            long long r = i;
            const int xx = (int)(r % v.w); r /= v.w;
            const int yy = (int)(r % v.h); r /= v.h;
            const int zz = (int)(r % v.d);
            const int b = (int)(r / v.d);
            s += bf(gz[v.at(b, zz, yy, xx) * ct + ch]);
        }
    }
    red[threadIdx.x] = row < rows ? s : 0.0f;
    __syncthreads();
    if (threadIdx.x < c) {
        float t = 0.0f;
        for (int k = 0; k < rows; ++k) t += red[k * c + threadIdx.x];
        atomicAdd(db + threadIdx.x, t);
    }
}

// ------------------------------------------------------ weight gradient ---
// dW[o][dz][dy][dx][c] += sum_v gz[v][o] x[v + (dz-1)P + (dy-1)(w+2) + dx-1][c]
// over padded voxels v of the interior span (gz is zero on halo voxels).
// Block (x: voxel chunk of one volume, y: (dz, dy), z: slice of the (dx, o, c)
// outputs); each thread accumulates a 2 (o) x 2 (c) block in FP32 over the
// chunk, staging 64 voxels of gz and 66 rows of x in shared memory at a time.
constexpr int kWgV = 64;

__global__ void __launch_bounds__(256) k_wgrad(const bf16 *__restrict__ gz, int g_ct, const bf16 *__restrict__ x,
                                               int x_ct, int x_co, int cin, int cout, float *__restrict__ dw,
                                               long long l0, long long span, long long lp, int w2, int p, int cpv,
                                               long long chunk)
{
    extern __shared__ float sm[];
    float *Gs = sm, *Xs = sm + kWgV * cout;
    const int dz = blockIdx.y / 3, dy = blockIdx.y % 3;
    const int nbo = cout / 2, nbc = cin / 2, nblk = 3 * nbo * nbc;
    const int blk = blockIdx.z * blockDim.x + threadIdx.x;
    const bool active = blk < nblk;
    const int dx = active ? blk / (nbo * nbc) : 0;
    const int rem = active ? blk % (nbo * nbc) : 0;
    const int ob = rem / nbc, cb = rem % nbc;
    float a00 = 0.0f, a01 = 0.0f, a10 = 0.0f, a11 = 0.0f;
    const int vol = blockIdx.x / cpv;
    const long long s0 = l0 + (long long)(blockIdx.x % cpv) * chunk;
    const long long s1 = std::min(s0 + chunk, l0 + span);
    const long long off = (long long)(dz - 1) * p + (long long)(dy - 1) * w2 - 1;
    const bf16 *gzv = gz + (long long)vol * lp * g_ct;
    const bf16 *xv = x + (long long)vol * lp * x_ct + x_co;
    for (long long v0 = s0; v0 < s1; v0 += kWgV) {
        __syncthreads();
        for (int i = threadIdx.x; i < kWgV * cout; i += blockDim.x) {
            const int vv = i / cout, o = i - vv * cout;
            const long long vg = v0 + vv;
            Gs[i] = vg < s1 ? bf(gzv[vg * g_ct + o]) : 0.0f;
        }
        for (int i = threadIdx.x; i < (kWgV + 2) * cin; i += blockDim.x) {
            const int rr = i / cin, c = i - rr * cin;
            const long long L = v0 + off + rr;
            Xs[i] = (L >= 0 && L < lp) ? bf(xv[L * x_ct + c]) : 0.0f;
        }
        __syncthreads();
        if (active) {
            const float *gp = Gs + 2 * ob;
            const float *xp = Xs + dx * cin + 2 * cb;
#pragma unroll 8
            for (int vv = 0; vv < kWgV; ++vv) {
                const float2 g = *reinterpret_cast<const float2 *>(gp + vv * cout);
                const float2 xx = *reinterpret_cast<const float2 *>(xp + vv * cin);
                a00 += g.x * xx.x;
                a01 += g.x * xx.y;
                a10 += g.y * xx.x;
                a11 += g.y * xx.y;
            }
        }
    }
    if (active) {
        const int tap = dz * 9 + dy * 3 + dx;
        float *d = dw + ((long long)(2 * ob) * 27 + tap) * cin + 2 * cb;
        atomicAdd(d, a00);
        atomicAdd(d + 1, a01);
        atomicAdd(d + 27ll * cin, a10);
        atomicAdd(d + 27ll * cin + 1, a11);
    }
}

// -------------------------------------------------- pooling, upsampling ---
// gradient of 2x2x2 max pooling, added to gx: each window's gradient goes to
// the first voxel in (dz, dy, dx) order that holds the window maximum
__global__ void k_pool2_back(const bf16 *__restrict__ x, int x_ct, int x_co, const bf16 *__restrict__ y, int y_ct,
                             const bf16 *__restrict__ gy, int gy_ct, bf16 *__restrict__ gx, int gx_ct, int gx_co,
                             int c, int n, VolIdx vo, VolIdx vi)
{
    const long long total = (long long)n * vo.d * vo.h * vo.w * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int xx = (int)(r % vo.w); r /= vo.w;
        const int yy = (int)(r % vo.h); r /= vo.h;
        const int zz = (int)(r % vo.d);
        const int b = (int)(r / vo.d);
        const long long ao = vo.at(b, zz, yy, xx);
        const float ymax = bf(y[ao * y_ct + ch]);
        const float g = bf(gy[ao * gy_ct + ch]);
        bool taken = false;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long ai = vi.at(b, 2 * zz + (k >> 2), 2 * yy + ((k >> 1) & 1), 2 * xx + (k & 1));
            const bool hit = !taken && bf(x[ai * x_ct + x_co + ch]) == ymax;
            taken |= hit;
            if (hit) {
                bf16 *t = gx + ai * gx_ct + gx_co + ch;
                *t = __float2bfloat16_rn(bf(*t) + g);
            }
        }
    }
}

// gradient of nearest 2x upsampling: gx[coarse] = sum of the 8 fine gradients
__global__ void k_up2_back(const bf16 *__restrict__ gy, int gy_ct, int gy_co, bf16 *__restrict__ gx, int gx_ct, int c,
                           int n, VolIdx vo, VolIdx vi)
{
    const long long total = (long long)n * vo.d * vo.h * vo.w * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int xx = (int)(r % vo.w); r /= vo.w;
        const int yy = (int)(r % vo.h); r /= vo.h;
        const int zz = (int)(r % vo.d);
        const int b = (int)(r / vo.d);
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            s += bf(gy[vi.at(b, 2 * zz + (k >> 2), 2 * yy + ((k >> 1) & 1), 2 * xx + (k & 1)) * gy_ct + gy_co + ch]);
        gx[vo.at(b, zz, yy, xx) * gx_ct + ch] = __float2bfloat16_rn(s);
    }
}

// ------------------------------------------------------------------ Adam ---
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       float wd)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
    }
}

// ------------------------------------------------------------------- host ---
lsm_status pack_layer(lsm_unet *u, int i, cudaStream_t st)
{
    const int ci = kLayers[i][0], co = kLayers[i][1];
    const float *w = u->params + layer_offset(i);
    lsm_conv3d *f = u->conv[i];
    lsm_conv3d *t = (u->train && i > 0) ? u->train->dconv[i] : nullptr;
    k_pack<<<grid_1d(27ll * ci * co), 256, 0, st>>>(w, ci, co, f->kc, t ? t->kc : 16, f->wimg, t ? t->wimg : nullptr,
                                                    w + 27ll * ci * co, f->bias);
    count_launch();
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

void train_free(UNetTrain *t)
{
    if (!t) return;
    cudaFree(t->grad);
    cudaFree(t->m);
    cudaFree(t->v);
    cudaFree(t->garena);
    cudaFree(t->loss);
    for (int i = 0; i < 14; ++i) conv_destroy(t->dconv[i]);
    free(t);
}

namespace {

lsm_vol sub_vol(const lsm_vol &v, int c_offset, int c)
{
    lsm_vol r = v;
    r.c_offset = c_offset;
    r.c = c;
    return r;
}

lsm_status train_alloc(lsm_unet *u, int n, int d, int h, int w, cudaStream_t st)
{
    const int64_t P = param_count();
    if (!u->train) {
        UNetTrain *t = (UNetTrain *)calloc(1, sizeof(UNetTrain));
        if (!t) return set_arg_error("lsm_unet_train_step: out of host memory");
        u->train = t;
        LSM_CUDA(cudaMalloc(&t->grad, P * 4));
        LSM_CUDA(cudaMalloc(&t->m, P * 4));
        LSM_CUDA(cudaMalloc(&t->v, P * 4));
        LSM_CUDA(cudaMalloc(&t->loss, 8));
        LSM_CUDA(cudaMemsetAsync(t->m, 0, P * 4, st));
        LSM_CUDA(cudaMemsetAsync(t->v, 0, P * 4, st));
        for (int i = 1; i < 14; ++i) {
            lsm_status rc = conv_alloc(kLayers[i][1], kLayers[i][0], 0, &t->dconv[i]);
            if (rc) return rc;
        }
        for (int i = 0; i < 14; ++i) {
            lsm_status rc = pack_layer(u, i, st);
            if (rc) return rc;
        }
    }
    UNetTrain *t = u->train;
    if (t->garena && t->n == n && t->d == d && t->h == h && t->w == w) return LSM_OK;
    LSM_CUDA(cudaStreamSynchronize(st));
    cudaFree(t->garena);
    t->garena = nullptr;
    const int zch[4] = {kW0, kW1, kW2, kW3};
    size_t off[NBUF + 4], total = 0;
    for (int b = 0; b < NBUF + 4; ++b) {
        const int L = b < NBUF ? kBufLevel[b] : b - NBUF;
        const int ch = b < NBUF ? kBufCh[b] : zch[L];
        off[b] = total;
        total += ((size_t)lsm_vol_bytes(n, d >> L, h >> L, w >> L, ch) + 255) / 256 * 256;
    }
    LSM_CUDA(cudaMalloc(&t->garena, total));
    LSM_CUDA(cudaMemsetAsync(t->garena, 0, total, st));
    for (int b = 0; b < NBUF + 4; ++b) {
        const int L = b < NBUF ? kBufLevel[b] : b - NBUF;
        const int ch = b < NBUF ? kBufCh[b] : zch[L];
        lsm_vol &v = b < NBUF ? t->g[b] : t->gz[L];
        v.data = (char *)t->garena + off[b];
        v.n = n; v.d = d >> L; v.h = h >> L; v.w = w >> L;
        v.c_total = ch; v.c_offset = 0; v.c = ch;
    }
    t->n = n; t->d = d; t->h = h; t->w = w;
    return LSM_OK;
}

// weight gradients on the tensor cores (wgrad_tc, default) or on the CUDA cores
int g_wgrad_tc = 1;

lsm_status wgrad(const lsm_vol &gz, const lsm_vol &x, int cin, int cout, float *dw, cudaStream_t st)
{
    const VolIdx v = vidx(x.d, x.h, x.w);
    const long long l0 = (long long)v.p + v.w2 + 1;
    const long long llast = (long long)x.d * v.p + (long long)x.h * v.w2 + x.w;
    const long long span = llast - l0 + 1;
    const int splits = (3 * (cout / 2) * (cin / 2) + 255) / 256;
    const long long base = 9ll * splits * x.n;
    long long cpv = std::max<long long>(1, std::min<long long>((span + kWgV - 1) / kWgV,
                                                               (8ll * sm_count() + base - 1) / base));
    long long chunk = (span + cpv - 1) / cpv;
    chunk = (chunk + kWgV - 1) / kWgV * kWgV;
    cpv = (span + chunk - 1) / chunk;
    const size_t smem = (size_t)(kWgV * cout + (kWgV + 2) * cin) * 4;
    static bool attr = false;
    if (!attr) {
        LSM_CUDA(cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 * 1024));
        attr = true;
    }
    const dim3 grid((unsigned)(cpv * x.n), 9, (unsigned)splits);
    k_wgrad<<<grid, 256, smem, st>>>((const bf16 *)gz.data, gz.c_total, (const bf16 *)x.data, x.c_total, x.c_offset,
                                     cin, cout, dw, l0, span, v.lp, v.w2, v.p, (int)cpv, chunk);
    count_launch();
    LSM_CUDA(cudaGetLastError());
    return LSM_OK;
}

}  // namespace

lsm_status train_step(lsm_unet *u, int n, int d, int h, int w, const float *dose, const float *rho,
                      const float *target, const lsm_adam_opts *opt, double *loss_host, cudaStream_t st)
{
    lsm_status rc = unet_buffers(u, n, d, h, w, st);
    if (rc) return rc;
    if ((rc = train_alloc(u, n, d, h, w, st))) return rc;
    UNetTrain *T = u->train;
    const int64_t P = param_count();
    LSM_CUDA(cudaMemsetAsync(T->grad, 0, P * 4, st));
    LSM_CUDA(cudaMemsetAsync(T->loss, 0, 8, st));
    if ((rc = unet_run(u, dose, rho, nullptr, st))) return rc;
    lsm_vol *V = u->vol, *G = T->g;
    const VolIdx v0 = vidx(d, h, w);
    const long long nvox = (long long)n * d * h * w;
    int tk = timer_begin(9, st);
    k_head_train<<<grid_1d(nvox), 256, 0, st>>>((const bf16 *)V[D0].data, V[D0].c_total, u->head, dose, target,
                                                u->dmax, (bf16 *)G[D0].data, G[D0].c_total,
                                                T->grad + layer_offset(14), T->loss, n, v0, 1.0f / (float)nvox);
    count_launch();
    timer_end(tk, st);
    LSM_CUDA(cudaGetLastError());

    auto back = [&](int i, const lsm_vol &gy, lsm_vol *gx) -> lsm_status {
        const int ci = kLayers[i][0], co = kLayers[i][1];
        const lsm_vol &yb = V[kConvOut[i]];
        const int L = kBufLevel[kConvOut[i]];
        const lsm_vol gz = sub_vol(T->gz[L], 0, co);
        const VolIdx vv = vidx(yb.d, yb.h, yb.w);
        const long long vox = (long long)n * yb.d * yb.h * yb.w;
        const int t0 = timer_begin(9, st);
        k_relu_mask<<<grid_1d(vox * (co / 8)), 256, 0, st>>>((const bf16 *)gy.data, gy.c_total, gy.c_offset,
                                                             (const bf16 *)yb.data, yb.c_total, 0, (bf16 *)gz.data,
                                                             gz.c_total, co / 8, n, vv);
        count_launch();
        const int rows = 256 / co;
        k_bias_grad<<<(unsigned)std::max<long long>(1, std::min<long long>((vox + rows - 1) / rows,
                                                                           4ll * sm_count())),
                      256, 0, st>>>((const bf16 *)gz.data, gz.c_total, co, n, vv,
                                    T->grad + layer_offset(i) + 27ll * ci * co);
        count_launch();
        lsm_status r = g_wgrad_tc ? wgrad_tc(gz, V[kConvIn[i]], ci, co, T->grad + layer_offset(i), st)
                                  : wgrad(gz, V[kConvIn[i]], ci, co, T->grad + layer_offset(i), st);
        timer_end(t0, st);
        if (r) return r;
        LSM_CUDA(cudaGetLastError());
        if (gx) return conv_forward(T->dconv[i], &gz, gx, 0, st);
        return LSM_OK;
    };
    auto up_back = [&](const lsm_vol &gy_fine, int c_off, int c, lsm_vol &gx) -> lsm_status {
        const VolIdx vo = vidx(gx.d, gx.h, gx.w), vi = vidx(gy_fine.d, gy_fine.h, gy_fine.w);
        const int t0 = timer_begin(9, st);
        k_up2_back<<<grid_1d((long long)n * gx.d * gx.h * gx.w * c), 256, 0, st>>>(
            (const bf16 *)gy_fine.data, gy_fine.c_total, c_off, (bf16 *)gx.data, gx.c_total, c, n, vo, vi);
        count_launch();
        timer_end(t0, st);
        LSM_CUDA(cudaGetLastError());
        return LSM_OK;
    };
    auto pool_back = [&](int skip, int pooled, int c) -> lsm_status {
        const lsm_vol &x = V[skip], &y = V[pooled];
        const VolIdx vo = vidx(y.d, y.h, y.w), vi = vidx(x.d, x.h, x.w);
        const int t0 = timer_begin(9, st);
        k_pool2_back<<<grid_1d((long long)n * y.d * y.h * y.w * c), 256, 0, st>>>(
            (const bf16 *)x.data, x.c_total, 0, (const bf16 *)y.data, y.c_total, (const bf16 *)G[pooled].data,
            G[pooled].c_total, (bf16 *)G[skip].data, G[skip].c_total, 0, c, n, vo, vi);
        count_launch();
        timer_end(t0, st);
        LSM_CUDA(cudaGetLastError());
        return LSM_OK;
    };
    lsm_vol gS0 = G[S0], gS1 = G[S1], gS2 = G[S2];
    if (!rc) rc = back(13, G[D0], &G[D0A]);
    if (!rc) rc = back(12, G[D0A], &gS0);
    if (!rc) rc = up_back(G[S0], kW0, kW0, G[D1]);
    if (!rc) rc = back(11, G[D1], &G[D1A]);
    if (!rc) rc = back(10, G[D1A], &gS1);
    if (!rc) rc = up_back(G[S1], kW1, kW1, G[D2]);
    if (!rc) rc = back(9, G[D2], &G[D2A]);
    if (!rc) rc = back(8, G[D2A], &gS2);
    if (!rc) rc = up_back(G[S2], kW2, kW2, G[B3]);
    if (!rc) rc = back(7, G[B3], &G[T3]);
    if (!rc) rc = back(6, G[T3], &G[P3]);
    if (!rc) rc = pool_back(S2, P3, kW2);
    if (!rc) rc = back(5, sub_vol(G[S2], 0, kW2), &G[T2]);
    if (!rc) rc = back(4, G[T2], &G[P2]);
    if (!rc) rc = pool_back(S1, P2, kW1);
    if (!rc) rc = back(3, sub_vol(G[S1], 0, kW1), &G[T1]);
    if (!rc) rc = back(2, G[T1], &G[P1]);
    if (!rc) rc = pool_back(S0, P1, kW0);
    if (!rc) rc = back(1, sub_vol(G[S0], 0, kW0), &G[T0]);
    if (!rc) rc = back(0, G[T0], nullptr);
    if (rc) return rc;
    if (opt && opt->lr > 0.0) {
        T->step += 1;
        const double c1 = 1.0 - pow(opt->beta1, (double)T->step), c2 = 1.0 - pow(opt->beta2, (double)T->step);
        tk = timer_begin(9, st);
        k_adam<<<grid_1d(P), 256, 0, st>>>(u->params, T->grad, T->m, T->v, P, (float)opt->lr, (float)opt->beta1,
                                           (float)opt->beta2, (float)opt->eps, (float)c1, (float)c2,
                                           (float)opt->weight_decay);
        count_launch();
        for (int i = 0; i < 14 && !rc; ++i) rc = pack_layer(u, i, st);
        timer_end(tk, st);
        if (rc) return rc;
    }
    if (loss_host) {
        LSM_CUDA(cudaMemcpyAsync(loss_host, T->loss, 8, cudaMemcpyDeviceToHost, st));
        unsigned err = 0;
        LSM_CUDA(cudaMemcpyAsync(&err, err_word(), 4, cudaMemcpyDeviceToHost, st));
        LSM_CUDA(cudaStreamSynchronize(st));
        if (err) {
            cudaMemsetAsync(err_word(), 0, 4, st);
            set_arg_error("lsm_unet_train_step: a tensor-core pipeline wait timed out");
            return LSM_ERR_TIMEOUT;
        }
    }
    return LSM_OK;
}

}  // namespace dn
}  // namespace lsm

using namespace lsm;

extern "C" {

lsm_status lsm_unet_train_step(lsm_unet *net, int32_t n, int32_t d, int32_t h, int32_t w, const float *dose,
                               const float *rho, const float *target, const lsm_adam_opts *opts, double *loss,
                               lsm_stream stream)
{
    if (!net || !dose || !rho || !target) return set_arg_error("lsm_unet_train_step: NULL argument");
    if (n < 1 || d < 8 || h < 8 || w < 8 || d % 8 || h % 8 || w % 8)
        return set_arg_error("lsm_unet_train_step: n >= 1 and d, h, w positive multiples of 8");
    if (opts && (opts->lr < 0.0 || opts->beta1 < 0.0 || opts->beta1 >= 1.0 || opts->beta2 < 0.0 ||
                 opts->beta2 >= 1.0 || opts->eps <= 0.0))
        return set_arg_error("lsm_unet_train_step: Adam options out of range");
    return dn::train_step(net, n, d, h, w, dose, rho, target, opts, loss, (cudaStream_t)stream);
}

lsm_status lsm_unet_params(const lsm_unet *net, float *dst, lsm_mem mem, lsm_stream stream)
{
    if (!net || !dst) return set_arg_error("lsm_unet_params: NULL argument");
    const cudaStream_t st = (cudaStream_t)stream;
    LSM_CUDA(cudaMemcpyAsync(dst, net->params, (size_t)dn::param_count() * 4,
                             mem == LSM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    if (mem == LSM_MEM_HOST) LSM_CUDA(cudaStreamSynchronize(st));
    return LSM_OK;
}

lsm_status lsm_unet_grad(const lsm_unet *net, float *dst, lsm_mem mem, lsm_stream stream)
{
    if (!net || !dst) return set_arg_error("lsm_unet_grad: NULL argument");
    if (!net->train) return set_arg_error("lsm_unet_grad: no training step yet");
    const cudaStream_t st = (cudaStream_t)stream;
    LSM_CUDA(cudaMemcpyAsync(dst, net->train->grad, (size_t)dn::param_count() * 4,
                             mem == LSM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    if (mem == LSM_MEM_HOST) LSM_CUDA(cudaStreamSynchronize(st));
    return LSM_OK;
}

lsm_status lsm_unet_set_wgrad(int tensor_cores)
{
    if (tensor_cores != 0 && tensor_cores != 1) return set_arg_error("lsm_unet_set_wgrad: 0 or 1");
    dn::g_wgrad_tc = tensor_cores;
    return LSM_OK;
}

}  // extern "C"
