// physics.cu -- interaction tables of the stated transport model, phantom set-up.
//
// The paper leaves the transport physics to its engine and fixes only the
// cutoffs (Sec. 2.3). The tables below implement the stated simplification
// from closed forms, evaluated in FP64 and stored as FP32 on a 1024-point
// log-energy grid (1 keV - 7 MeV):
//   Compton:      Klein-Nishina total cross section per electron x electrons/g;
//   photoelectric C_pe Z^3 / E^3 per electron, C_pe such that the photoelectric
//                 and Compton coefficients of water are equal at 30 keV;
//   pair:         C_pp Z (E - 2 m c^2) / E per electron above threshold, C_pp
//                 such that pair is 5% of the total coefficient of water at 6 MeV;
//   stopping:     Bethe collision stopping power of electrons, no density effect.
// Material classes: 0 water-like (Z 7.4, 3.34e23 e/g, I 75 eV), 1 bone
// (Z 13.8, 0.96 x 3.34e23 e/g, I 106.4 eV).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "handles.cuh"

namespace lsm {
namespace {

constexpr double kRe = 2.8179403262e-13;   // classical electron radius, cm
__constant__ double c_ne[2] = {3.34e23, 3.34e23 * 0.96};
__constant__ double c_z[2] = {7.4, 13.8};
__constant__ double c_iev[2] = {75.0, 106.4};

__device__ double kn_total(double E)
{
    const double k = E / kMeD, a = 1.0 + 2.0 * k, L = log(a);
    return 2.0 * kPiD * kRe * kRe *
           ((1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k) + L / (2.0 * k) - (1.0 + 3.0 * k) / (a * a));
}

__device__ double photo_per_e(double E, double Z)
{
    const double cpe = kn_total(0.03) * (0.03 * 0.03 * 0.03) / (7.4 * 7.4 * 7.4);
    return cpe * Z * Z * Z / (E * E * E);
}

__device__ double pair_per_e(double E, double Z)
{
    if (!(E > 2.0 * kMeD)) return 0.0;
    const double s6 = (0.05 / 0.95) * (kn_total(6.0) + photo_per_e(6.0, 7.4));
    const double cpp = s6 * 6.0 / (7.4 * (6.0 - 2.0 * kMeD));
    return cpp * Z * (E - 2.0 * kMeD) / E;
}

__device__ double bethe(double E, int m)
{
    const double tau = E / kMeD, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    const double im = c_iev[m] * 1e-6 / kMeD;
    const double F = 1.0 - b2 + (tau * tau / 8.0 - (2.0 * tau + 1.0) * log(2.0)) / (g * g);
    return 2.0 * kPiD * kRe * kRe * kMeD * c_ne[m] / b2 * (log(tau * tau * (tau + 2.0) / (2.0 * im * im)) + F);
}

__global__ void k_tables(float4 *__restrict__ xs, double *__restrict__ mutot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * kGrid) return;
    const int m = i / kGrid, j = i % kGrid;
    const double dl = (kLnEmax - kLnEmin) / (kGrid - 1);
    const double E = exp(kLnEmin + j * dl);
    const double c = c_ne[m] * kn_total(E), p = c_ne[m] * photo_per_e(E, c_z[m]),
                 q = c_ne[m] * pair_per_e(E, c_z[m]);
    xs[i] = make_float4((float)c, (float)p, (float)q, (float)bethe(E, m));
    mutot[i] = c + p + q;
}

// integral of the Klein-Nishina density of eta = E/E' from 1 to eta (up to a
// constant factor), k = E/mc^2:  f(t) = t^-2 (1/t + t - sin^2 theta),
// cos theta = 1 - (t - 1)/k
__device__ double kn_cdf(double eta, double k)
{
    const double ie = 1.0 / eta, le = log(eta), k1 = k + 1.0;
    return 0.5 * (1.0 - ie * ie) + le + ie - 1.0 + (k1 * k1 * (1.0 - ie) - 2.0 * k1 * le + eta - 1.0) / (k * k);
}

// inverse CDF table, v = (eta - 1) / (2k), by bisection in FP64
__global__ void k_kn_table(float *__restrict__ tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kKnE * kKnU) return;
    const int ie = i / kKnU, ju = i % kKnU;
    const double E = exp(kKnLnE0 + ie * ((kKnLnE1 - kKnLnE0) / (kKnE - 1)));
    const double k = E / kMeD, emax = 1.0 + 2.0 * k;
    const double target = ((double)ju / (kKnU - 1)) * kn_cdf(emax, k);
    double lo = 1.0, hi = emax;
    for (int it = 0; it < 64; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (kn_cdf(mid, k) < target) lo = mid; else hi = mid;
    }
    double v = (0.5 * (lo + hi) - 1.0) / (2.0 * k);
    if (ju == 0) v = 0.0;
    if (ju == kKnU - 1) v = 1.0;
    tab[i] = (float)v;
}

__global__ void k_rho_max(const float *__restrict__ rho, const uint8_t *__restrict__ mat, int64_t n,
                          unsigned *__restrict__ bits)
{
    __shared__ unsigned s[2];
    if (threadIdx.x < 2) s[threadIdx.x] = 0u;
    __syncthreads();
    unsigned loc[2] = {0u, 0u};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned b = __float_as_uint(rho[i]);     // non-negative floats order as integers
        const int m = mat[i] ? 1 : 0;
        loc[m] = b > loc[m] ? b : loc[m];
    }
    atomicMax(&s[0], loc[0]);
    atomicMax(&s[1], loc[1]);
    __syncthreads();
    if (threadIdx.x < 2) atomicMax(&bits[threadIdx.x], s[threadIdx.x]);
}

// majorant: max over material classes of (largest density) x mu_total, with a
// 2^-16 relative margin so FP32 rounding never puts mu above it
__global__ void k_majorant(const double *__restrict__ mutot, const unsigned *__restrict__ bits,
                           float *__restrict__ mumax)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kGrid) return;
    const double r0 = (double)__uint_as_float(bits[0]), r1 = (double)__uint_as_float(bits[1]);
    const double v = fmax(r0 * mutot[j], r1 * mutot[kGrid + j]);
    mumax[j] = (float)(v * (1.0 + 1.0 / 65536.0));
}

__global__ void k_rhomat(const float *__restrict__ rho, const uint8_t *__restrict__ mat, int64_t n, double vol,
                         float *__restrict__ rhomat, double *__restrict__ inv_mass)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float r = rho[i];
        rhomat[i] = mat[i] ? -r : r;
        inv_mass[i] = 1.0 / ((double)r * vol);
    }
}

__global__ void k_check_phantom(const float *__restrict__ rho, const uint8_t *__restrict__ mat, int64_t n,
                                unsigned *__restrict__ bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float r = rho[i];
        if (!(r >= 1e-4f && r <= 25.0f) || mat[i] > 1) atomicOr(bad, 1u);
    }
}

}  // namespace

// The phantom's memory returns to the pool in the order of the legacy
// default stream.
void free_phantom(lsm_phantom *P)
{
    if (!P) return;
    dev_free(P->d_rho);
    dev_free(P->d_mat);
    dev_free(P->d_rhomat);
    dev_free(P->d_inv_mass);
    dev_free(P->d_xs);
    dev_free(P->d_mumax);
    dev_free(P->d_flags);
    free(P);
}

namespace {
// The cross-section and inverse Klein-Nishina tables depend on no phantom:
// computed once per device and copied into each phantom.
struct SharedTables {
    float4 *xs = nullptr;        // [2][kGrid]
    double *mutot = nullptr;     // [2][kGrid]
    float *kn = nullptr;         // [kKnE][kKnU]
};
std::mutex g_tab_m;
SharedTables g_tab[64];

cudaError_t shared_tables(cudaStream_t st, SharedTables **out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_tab_m);
    SharedTables &T = g_tab[dev];
    if (!T.xs) {
        SharedTables n;
        cudaError_t e = cudaMalloc(&n.xs, 2 * kGrid * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc(&n.mutot, 2 * kGrid * 8);
        if (e == cudaSuccess) e = cudaMalloc(&n.kn, kKnE * kKnU * 4);
        if (e == cudaSuccess) {
            k_tables<<<(2 * kGrid + 127) / 128, 128, 0, st>>>(n.xs, n.mutot);
            count_launch();
            k_kn_table<<<(kKnE * kKnU + 127) / 128, 128, 0, st>>>(n.kn);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFree(n.xs); cudaFree(n.mutot); cudaFree(n.kn);
            return e;
        }
        T = n;
    }
    *out = &T;
    return cudaSuccess;
}
}  // namespace

lsm_status create_phantom(const lsm_phantom_desc *D, lsm_phantom **out, cudaStream_t st, bool deferred)
{
    if (!D || !out || !D->rho || !D->mat) return set_arg_error("lsm_phantom_create: NULL argument");
    *out = nullptr;
    if (D->nx < 1 || D->ny < 1 || D->nz < 1 || D->nx > 4096 || D->ny > 4096 || D->nz > 4096)
        return set_arg_error("lsm_phantom_create: dimensions must be 1..4096");
    if (!(D->dx > 0) || !(D->dy > 0) || !(D->dz > 0) || !isfinite(D->x0) || !isfinite(D->y0) || !isfinite(D->z0))
        return set_arg_error("lsm_phantom_create: voxel sizes must be > 0");
    const int64_t n = (int64_t)D->nx * D->ny * D->nz;
    if (n >= ((int64_t)1 << 31)) return set_arg_error("lsm_phantom_create: more than 2^31 voxels");
    lsm_phantom *P = (lsm_phantom *)calloc(1, sizeof(lsm_phantom));
    if (!P) return set_arg_error("lsm_phantom_create: out of host memory");
    P->uid = next_uid();
    cudaGetDevice(&P->device);
    P->nx = D->nx; P->ny = D->ny; P->nz = D->nz;
    P->dx = D->dx; P->dy = D->dy; P->dz = D->dz; P->x0 = D->x0; P->y0 = D->y0; P->z0 = D->z0;
    cudaError_t e;
    double *d_mutot = nullptr;
    unsigned *d_bits = nullptr;
    const cudaMemcpyKind kind = D->mem == LSM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    unsigned bits[3] = {0, 0, 0};
#define CK(call)                                                                        \
    do {                                                                                \
        e = (call);                                                                     \
        if (e != cudaSuccess) {                                                         \
            cudaStreamSynchronize(st); free_phantom(P);                                 \
            return set_cuda_error(e, #call);                                            \
        }                                                                               \
    } while (0)
#define CKL(name) do { count_launch(); CK(cudaGetLastError()); } while (0)
    SharedTables *tab = nullptr;
    CK(shared_tables(st, &tab));
    d_mutot = tab->mutot;
    CK(dev_malloc((void **)&P->d_rho, n * 4, st));
    CK(dev_malloc((void **)&P->d_mat, n, st));
    CK(dev_malloc((void **)&P->d_rhomat, n * 4, st));
    CK(dev_malloc((void **)&P->d_inv_mass, n * 8, st));
    CK(dev_malloc((void **)&P->d_xs, 2 * kGrid * sizeof(float4), st));
    // majorant followed by the inverse-KN table: staged into shared memory by one copy
    CK(dev_malloc((void **)&P->d_mumax, kGrid * 4 + kKnE * kKnU * 4, st));
    CK(dev_malloc((void **)&P->d_flags, 16, st));
    d_bits = P->d_flags;
    CK(cudaMemcpyAsync(P->d_rho, D->rho, n * 4, kind, st));
    CK(cudaMemcpyAsync(P->d_mat, D->mat, n, kind, st));
    CK(cudaMemsetAsync(d_bits, 0, 16, st));
    const int g = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_check_phantom<<<g, 256, 0, st>>>(P->d_rho, P->d_mat, n, d_bits + 2);
    CKL("k_check_phantom");
    k_rho_max<<<g, 256, 0, st>>>(P->d_rho, P->d_mat, n, d_bits);
    CKL("k_rho_max");
    k_rhomat<<<g, 256, 0, st>>>(P->d_rho, P->d_mat, n, D->dx * D->dy * D->dz, P->d_rhomat, P->d_inv_mass);
    CKL("k_rhomat");
    CK(cudaMemcpyAsync(P->d_xs, tab->xs, 2 * kGrid * sizeof(float4), cudaMemcpyDeviceToDevice, st));
    k_majorant<<<(kGrid + 127) / 128, 128, 0, st>>>(d_mutot, d_bits, P->d_mumax);
    CKL("k_majorant");
    CK(cudaMemcpyAsync(P->d_mumax + kGrid, tab->kn, kKnE * kKnU * 4, cudaMemcpyDeviceToDevice, st));
    if (deferred) {
        // the check's verdict stays on the device: the transport kernels skip
        // an invalid phantom, and lsm_dose to host memory or
        // lsm_phantom_check report it
        P->validated = 0;
        *out = P;
        return LSM_OK;
    }
    CK(cudaMemcpyAsync(bits, d_bits, 12, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    P->validated = 1;
    if (bits[2]) {
        free_phantom(P);
        return set_arg_error("lsm_phantom_create: densities must be in [1e-4, 25] and materials in {0, 1}");
    }
    float rf[2];
    memcpy(rf, bits, 8);
    P->rho_max[0] = rf[0];
    P->rho_max[1] = rf[1];
    *out = P;
    return LSM_OK;
#undef CK
#undef CKL
}

}  // namespace lsm
