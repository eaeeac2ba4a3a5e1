// unet.cuh -- shared state of the denoiser (inference in denoise.cu, training
// in train.cu): padded-volume indexing, the network's layer table, the layer
// and network handles.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

// Layers whose three dx taps share one MMA (N = 3 cout): cout <= 64 and at
// least 32 input channels per stage. With 16 channels per stage the twelve
// small boxes per stage this needs cost more than the MMAs they save
// (measured on the 16-channel layers at 128^3).
__host__ __device__ constexpr bool conv_fused(int cout, int kc) { return cout <= 64 && kc >= 32; }

// Element offset of weight (output channel n, input channel chunk * kc + k,
// tap dz, dy, dx) in a layer's BF16 operand image. The image holds, per
// (channel chunk, dz), the stage's 9 taps x cout x kc weights in the K-major
// core-matrix layout of the MMA's B operand (8 rows x 8 K elements of 16
// bytes; rows step 128 bytes per 8-row group, the two 8-element K halves of
// a 16-wide K step are n_rows x 16 bytes apart). Fused layers (conv_fused)
// put the three dx taps of one (dz, dy) side by side as one operand of
// 3 cout rows (row dx cout + n), so that one MMA covers them.
__host__ __device__ __forceinline__ size_t wimg_offset(int cout, int kc, int chunk, int dz, int dy, int dx, int n,
                                                       int k)
{
    if (conv_fused(cout, kc)) {
        const size_t blk = (size_t)((chunk * 3 + dz) * 3 + dy) * 3 * cout * kc;
        const int rows = 3 * cout, r = dx * cout + n;
        return blk + (size_t)(k / 8) * rows * 8 + (size_t)(r / 8) * 64 + (r % 8) * 8 + (k % 8);
    }
    const size_t blk = (size_t)((chunk * 3 + dz) * 9 + dy * 3 + dx) * cout * kc;
    return blk + (size_t)(k / 8) * cout * 8 + (size_t)(n / 8) * 64 + (n % 8) * 8 + (k % 8);
}

struct lsm_conv3d {
    int cin, cout, relu, kc;
    __nv_bfloat16 *wimg;      // packed operand images [cin/kc][dz][9 taps][cout x kc]
    float *bias;              // [cout], values rounded to BF16
};

namespace lsm {
namespace dn {

// index of interior voxel (z, y, x) of volume b in a padded volume
struct VolIdx {
    int d, h, w;
    long long lp;             // padded voxels per volume
    int w2, p;                // w + 2, (h + 2)(w + 2)
    __host__ __device__ long long at(int b, int z, int y, int x) const
    {
        return (long long)b * lp + (long long)(z + 1) * p + (long long)(y + 1) * w2 + x + 1;
    }
};

__host__ __device__ inline VolIdx vidx(int d, int h, int w)
{
    VolIdx v;
    v.d = d; v.h = h; v.w = w;
    v.w2 = w + 2;
    v.p = (h + 2) * (w + 2);
    v.lp = (long long)(d + 2) * v.p;
    return v;
}

// ---- network: widths 16/32/64/128, four levels ----
constexpr int kW0 = 16, kW1 = 32, kW2 = 64, kW3 = 128;
constexpr int kInCh = 16;
// (c_in, c_out) of the 14 conv layers in network order
constexpr int kLayers[14][2] = {{kInCh, kW0},   {kW0, kW0}, {kW0, kW1}, {kW1, kW1}, {kW1, kW2},
                                {kW2, kW2},     {kW2, kW3}, {kW3, kW2}, {2 * kW2, kW2}, {kW2, kW1},
                                {2 * kW1, kW1}, {kW1, kW0}, {2 * kW0, kW0}, {kW0, kW0}};
enum Buf { X0, T0, S0, P1, T1, S1, P2, T2, S2, P3, T3, B3, D2A, D2, D1A, D1, D0A, D0, NBUF };
constexpr int kBufLevel[NBUF] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 1, 1, 0, 0};
constexpr int kBufCh[NBUF] = {kInCh, kW0, 2 * kW0, kW0, kW1, 2 * kW1, kW1, kW2, 2 * kW2, kW2, kW3, kW2,
                              kW2,   kW1, kW1,     kW0, kW0, kW0};
// conv layer i reads all channels of buffer kConvIn[i] and writes channels
// [0, c_out) of buffer kConvOut[i]
constexpr int kConvIn[14] = {X0, T0, P1, T1, P2, T2, P3, T3, S2, D2A, S1, D1A, S0, D0A};
constexpr int kConvOut[14] = {T0, S0, T1, S1, T2, S2, T3, B3, D2A, D2, D1A, D1, D0A, D0};

inline int64_t layer_offset(int i)
{   // first parameter of layer i in the flat vector (weights, then bias)
    int64_t n = 0;
    for (int k = 0; k < i; ++k) n += 27ll * kLayers[k][0] * kLayers[k][1] + kLayers[k][1];
    return n;
}
inline int64_t param_count() { return layer_offset(14) + kW0 + 1; }

lsm_status check_vol(const lsm_vol *v, const char *what);
lsm_status conv_forward(const lsm_conv3d *cv, const lsm_vol *in, const lsm_vol *out, int ctas_per_sm,
                        cudaStream_t st);
lsm_status conv_alloc(int cin, int cout, int relu, lsm_conv3d **out);
lsm_status conv_create(int cin, int cout, int relu, const float *w, const float *b, lsm_conv3d **out,
                       cudaStream_t st);
void conv_destroy(lsm_conv3d *cv);
int kc_for(int cin, int cout);
lsm_status pool_or_up(const lsm_vol *in, const lsm_vol *out, bool up, cudaStream_t st);
int grid_1d(long long work);
unsigned *err_word();
lsm_status wgrad_tc(const lsm_vol &gz, const lsm_vol &x, int cin, int cout, float *dw, cudaStream_t st);

}  // namespace dn
}  // namespace lsm

// training state (allocated by the first training step)
struct UNetTrain {
    float *grad, *m, *v;          // [param_count]
    lsm_conv3d *dconv[14];        // data-gradient layers: mirrored, channel-transposed weights
    void *garena;                 // gradient volumes and per-level scratch
    lsm_vol g[lsm::dn::NBUF];     // gradient of each activation buffer
    lsm_vol gz[4];                // ReLU-masked output gradient, per level (widest layer)
    double *loss;                 // device accumulator
    int n, d, h, w;               // shape of the gradient buffers
    long long step;
};

struct lsm_unet {
    lsm_conv3d *conv[14];
    float *params;                // device FP32 parameters, flat (master copy)
    float *head;                  // = params + layer_offset(14): 16 weights and the bias
    int n, d, h, w;               // shape the activation buffers are allocated for
    void *arena;
    lsm_vol vol[lsm::dn::NBUF];
    unsigned *dmax;               // [n] FP32 bits
    float *io;                    // device staging for host calls: dose, rho, out
    size_t io_cap;
    UNetTrain *train;
    // the layers between input packing and the output head (convolutions,
    // pooling, upsampling) touch only the activation buffers: captured once
    // per buffer allocation as a CUDA graph and replayed
    void *gexec;                  // cudaGraphExec_t, or null
    int g_warm;                   // 1: a direct pass has run on these buffers (one-time set-up done);
                                  // -1: capture failed, launch directly
    int64_t g_kernels;            // kernels in the graph
};

namespace lsm {
namespace dn {
lsm_status unet_buffers(lsm_unet *u, int n, int d, int h, int w, cudaStream_t st);
void unet_drop_graph(lsm_unet *u);
lsm_status unet_run(lsm_unet *u, const float *dose, const float *rho, float *out, cudaStream_t st);
lsm_status pack_layer(lsm_unet *u, int i, cudaStream_t st);
void train_free(UNetTrain *t);
}  // namespace dn
}  // namespace lsm
