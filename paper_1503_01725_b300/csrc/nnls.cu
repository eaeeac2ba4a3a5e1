// nnls.cu -- the commissioning problem of Eq. 8 in FP64 on the GPU.
//
//   min_{x >= 0} F(x) = ||A x - b||^2
//
// k_gram forms G = A^T A and c = A^T b (FP64 CUDA cores). Two solvers then run
// in one CTA of 1024 threads with G resident in L2:
//   * active set (Lawson & Hanson 1974): the passive-set least squares is
//     solved through a Cholesky factor of G restricted to the passive set,
//     updated as variables enter or leave (O(k^2) per change);
//   * gradient projection with Armijo's rule (Sec. 2.2.4):
//     x <- max(0, x - s grad F), s = s_bar beta^j for the first j with
//     F(x_new) <= F(x) + sigma grad F . (x_new - x); stop when the relative
//     change of F is below delta. The decrease F(x_new) - F(x) is evaluated as
//     g.d + d^T G d (d = x_new - x) so that no large terms cancel.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "handles.cuh"

namespace lsm {
namespace {

constexpr int kT = 1024;

__global__ void k_gram(const double *__restrict__ A, const double *__restrict__ b, int m, int n,
                       double *__restrict__ G, double *__restrict__ c)
{
    __shared__ double ta[32][33], tb[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    double acc[4] = {0, 0, 0, 0};
    double accb = 0.0;
    for (int r0 = 0; r0 < m; r0 += 32) {
        for (int q = ty; q < 32; q += 8) {
            const int r = r0 + q;
            ta[q][tx] = (r < m && i0 + tx < n) ? A[(size_t)r * n + i0 + tx] : 0.0;
            tb[q][tx] = (r < m && j0 + tx < n) ? A[(size_t)r * n + j0 + tx] : 0.0;
        }
        __syncthreads();
        for (int q = 0; q < 32; ++q) {
            const double bj = tb[q][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += ta[q][ty + 8 * k] * bj;
        }
        if (blockIdx.x == 0 && ty == 0) {
            for (int q = 0; q < 32 && r0 + q < m; ++q) accb += ta[q][tx] * b[r0 + q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = i0 + ty + 8 * k, j = j0 + tx;
        if (i < n && j < n) G[(size_t)i * n + j] = acc[k];
    }
    if (blockIdx.x == 0 && ty == 0 && i0 + tx < n) c[i0 + tx] = accb;
}

// ---- block helpers (1024 threads) ----
__device__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = red[l];
        t = warp_sum(t);
        if (l == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Three block-wide sums in one pass (red: at least 97 doubles).
__device__ void block_sum3(double &a, double &b, double &c, double *red)
{
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { red[w] = a; red[32 + w] = b; red[64 + w] = c; }
    __syncthreads();
    if (w == 0) {
        const double ta = warp_sum(red[l]), tb = warp_sum(red[32 + l]), tc = warp_sum(red[64 + l]);
        if (l == 0) { red[96] = ta; red[97] = tb; red[98] = tc; }
    }
    __syncthreads();
    a = red[96]; b = red[97]; c = red[98];
}

// argmax of v over j with mask(j) true; returns index (-1 if none) and value
__device__ int block_argmax(double v, int j, double *redv, int *redi, double *best)
{
    // warp stage
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (ov > v || (ov == v && oj >= 0 && (j < 0 || oj < j))) { v = ov; j = oj; }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { redv[w] = v; redi[w] = j; }
    __syncthreads();
    if (w == 0) {
        v = redv[l]; j = redi[l];
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oj = __shfl_xor_sync(0xffffffffu, j, o);
            if (ov > v || (ov == v && oj >= 0 && (j < 0 || oj < j))) { v = ov; j = oj; }
        }
        if (l == 0) { redv[32] = v; redi[32] = j; }
    }
    __syncthreads();
    *best = redv[32];
    return redi[32];
}

struct NnlsOut {
    int iterations, converged, status;   // status 0 ok, 1 not converged, 2 numerical failure
    double objective;
};

// The passive set's factor: G[P,P] = L L^T for P = ord[0..k) in the order
// the variables entered, L lower triangular, column-major with leading
// dimension n (element (i, j), i >= j, at L[j n + i]); invd[i] = 1 / L(i, i).
// Lawson and Hanson's iteration adds or drops one variable at a time, so the
// factor is extended by one row (a forward substitution) or has a row and
// column deleted (a rank-one update of the trailing block, Givens form) in
// O(k^2) instead of being refactored in O(k^3). The triangular work runs on
// one warp; only warp-level synchronisation is needed inside it.

// Column j of the factor, indexable by row i >= j. Packed (shared memory):
// the lower triangle column after column, column j holding rows j..n-1;
// otherwise (global memory) leading dimension n.
template <bool PK>
__device__ __forceinline__ double *lcol(double *L, int n, int j)
{
    return PK ? L + (size_t)j * n - (size_t)j * (j + 1) / 2 : L + (size_t)j * n;
}

// r <- L^-1 r over the first k entries
template <bool PK>
__device__ void warp_forward(double *__restrict__ L, int n, int k, const double *invd, double *r)
{
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < k; ++j) {
        const double rj = r[j] * invd[j];
        __syncwarp();
        if (lane == 0) r[j] = rj;
        const double *col = lcol<PK>(L, n, j);
        for (int i = j + 1 + lane; i < k; i += 32) r[i] -= col[i] * rj;
        __syncwarp();
    }
}

// z <- L^-T y over the first k entries
template <bool PK>
__device__ void warp_backward(double *__restrict__ L, int n, int k, const double *invd, const double *y, double *z)
{
    const int lane = threadIdx.x & 31;
    for (int i = k - 1; i >= 0; --i) {
        const double *col = lcol<PK>(L, n, i);
        double s = 0.0;
        for (int l = i + 1 + lane; l < k; l += 32) s += col[l] * z[l];
        s = warp_sum(s);
        if (lane == 0) z[i] = (y[i] - s) * invd[i];
        __syncwarp();
    }
}

// Append variable t (position k); false when G restricted to P + {t} is not
// positive definite (the new pivot is not > 0). r: scratch of k doubles.
template <bool PK>
__device__ bool warp_add(const double *__restrict__ G, double *L, int n, int k, int *ord, double *invd, int t,
                         double *r)
{
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < k; i += 32) r[i] = G[(size_t)ord[i] * n + t];
    __syncwarp();
    warp_forward<PK>(L, n, k, invd, r);
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s += r[i] * r[i];
    s = warp_sum(s);
    const double d = G[(size_t)t * n + t] - s;
    if (!(d > 0.0)) return false;
    for (int j = lane; j < k; j += 32) lcol<PK>(L, n, j)[k] = r[j];
    if (lane == 0) {
        const double dd = sqrt(d);
        lcol<PK>(L, n, k)[k] = dd;
        invd[k] = 1.0 / dd;
        ord[k] = t;
    }
    __syncwarp();
    return true;
}

// Drop position q of k: delete row and column q, then restore the trailing
// block's factor with the rank-one update L33 L33^T + v v^T, v the deleted
// column below the diagonal. v: scratch of k doubles.
template <bool PK>
__device__ void warp_remove(double *L, int n, int k, int *ord, double *invd, int q, double *v)
{
    const int lane = threadIdx.x & 31;
    const int m = k - 1 - q;
    for (int i = lane; i < m; i += 32) v[i] = lcol<PK>(L, n, q)[q + 1 + i];
    __syncwarp();
    for (int j = 0; j < q; ++j) {          // columns left of q lose row q
        double *col = lcol<PK>(L, n, j);
        for (int i0 = q + 1; i0 < k; i0 += 32) {
            const int i = i0 + lane;
            const double val = i < k ? col[i] : 0.0;
            __syncwarp();
            if (i < k) col[i - 1] = val;
            __syncwarp();
        }
    }
    for (int j = q + 1; j < k; ++j) {      // columns right of q move up and left
        const double *src = lcol<PK>(L, n, j);
        double *dst = lcol<PK>(L, n, j - 1);
        for (int i = j + lane; i < k; i += 32) dst[i - 1] = src[i];
        __syncwarp();
    }
    if (lane == 0)
        for (int p = q; p + 1 < k; ++p) ord[p] = ord[p + 1];
    __syncwarp();
    for (int c = 0; c < m; ++c) {          // Givens form of the rank-one update
        double *col = lcol<PK>(L, n, q + c);
        const double lcc = col[q + c], vc = v[c];
        const double r = sqrt(lcc * lcc + vc * vc);
        const double ics = lcc / r, sn = vc / lcc, cs = r / lcc;
        __syncwarp();
        if (lane == 0) {
            col[q + c] = r;
            invd[q + c] = 1.0 / r;
        }
        for (int i = c + 1 + lane; i < m; i += 32) {
            const double lic = (col[q + i] + sn * v[i]) * ics;
            col[q + i] = lic;
            v[i] = cs * v[i] - sn * lic;
        }
        __syncwarp();
    }
}

// PK: the factor packed in shared memory after the other arrays (when it
// fits); otherwise in the global scratch Lg (n x n).
template <bool PK>
__global__ void __launch_bounds__(kT) k_lawson_hanson(const double *__restrict__ G, const double *__restrict__ cg,
                                                      int n, double tol_scale, int max_iter, double *__restrict__ Lg,
                                                      double *__restrict__ xout, NnlsOut *out)
{
    extern __shared__ double sm[];
    double *x = sm, *w = sm + n, *z = sm + 2 * n, *y = sm + 3 * n, *c = sm + 4 * n, *invd = sm + 5 * n,
           *zf = sm + 6 * n;
    int *P = (int *)(sm + 7 * n), *ord = P + n;
    double *L = PK ? sm + 8 * n : Lg;       // 7 n doubles + 2 n ints = 8 n doubles
    __shared__ double red[33];
    __shared__ int redi[33];
    __shared__ int s_k, s_status;
    const bool w0 = threadIdx.x < 32;
    for (int j = threadIdx.x; j < n; j += kT) { x[j] = 0.0; P[j] = 0; c[j] = cg[j]; w[j] = cg[j]; }
    if (threadIdx.x == 0) { s_status = 0; s_k = 0; }
    // tolerance 10 eps ||G||_1 max(m, n) (Lawson & Hanson's test on the dual)
    double cmax = 0.0;
    for (int j = threadIdx.x; j < n; j += kT) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(G[(size_t)i * n + j]);
        cmax = fmax(cmax, s);
    }
    for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int q = 0; q < 32; ++q) v = fmax(v, red[q]);
        red[32] = v;
    }
    __syncthreads();
    const double tol = tol_scale * red[32];
    __syncthreads();
    int it = 0;
    for (;;) {
        // most positive gradient component outside the passive set
        double bv = -INFINITY;
        int bj = -1;
        for (int j = threadIdx.x; j < n; j += kT)
            if (!P[j] && (w[j] > bv || (w[j] == bv && bj >= 0 && j < bj) || bj < 0)) { bv = w[j]; bj = j; }
        double best;
        const int t = block_argmax(bj >= 0 ? bv : -INFINITY, bj, red, redi, &best);
        if (t < 0 || !(best > tol) || it >= max_iter) break;
        if (w0) {
            const int k = s_k;
            const bool ok = warp_add<PK>(G, L, n, k, ord, invd, t, y);
            if (threadIdx.x == 0) {
                if (ok) { P[t] = 1; s_k = k + 1; }
                else s_status = 2;
            }
        }
        __syncthreads();
        if (s_status) break;
        for (;;) {
            ++it;
            const int k = s_k;
            for (int j = threadIdx.x; j < n; j += kT) z[j] = 0.0;
            __syncthreads();
            if (w0) {   // z_P = G[P,P]^-1 c_P through the factor
                for (int i = threadIdx.x; i < k; i += 32) y[i] = c[ord[i]];
                __syncwarp();
                warp_forward<PK>(L, n, k, invd, y);
                warp_backward<PK>(L, n, k, invd, y, zf);
                for (int i = threadIdx.x; i < k; i += 32) z[ord[i]] = zf[i];
            }
            __syncthreads();
            // all passive z positive?
            int bad = 0;
            for (int q = threadIdx.x; q < k; q += kT) bad |= !(z[ord[q]] > 0.0);
            bad = __syncthreads_or(bad);
            if (!bad) {
                for (int j = threadIdx.x; j < n; j += kT) x[j] = z[j];
                __syncthreads();
                break;
            }
            double a = INFINITY;
            for (int q = threadIdx.x; q < k; q += kT) {
                const int j = ord[q];
                if (!(z[j] > 0.0)) a = fmin(a, x[j] / (x[j] - z[j]));
            }
            for (int o = 16; o > 0; o >>= 1) a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
            __syncthreads();
            if (threadIdx.x < 32) {
                double v = red[threadIdx.x];
                for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (threadIdx.x == 0) red[32] = v;
            }
            __syncthreads();
            const double alpha = red[32];
            for (int j = threadIdx.x; j < n; j += kT) {
                x[j] = x[j] + alpha * (z[j] - x[j]);
                if (P[j] && !(x[j] > tol)) P[j] = 0;
                if (!P[j]) x[j] = 0.0;
            }
            __syncthreads();
            if (w0) {   // drop the variables that left P from the factor, last position first
                int kk = k;
                for (int q = k - 1; q >= 0; --q)
                    if (!P[ord[q]]) { warp_remove<PK>(L, n, kk, ord, invd, q, y); --kk; }
                if (threadIdx.x == 0) s_k = kk;
            }
            __syncthreads();
            if (it >= max_iter) break;
        }
        if (s_status) break;
        // w = c - G x, x zero outside P (G symmetric: row ord[q] read along j)
        {
            const int k = s_k;
            for (int j = threadIdx.x; j < n; j += kT) {
                double s = 0.0;
                for (int q = 0; q < k; ++q) {
                    const int l = ord[q];
                    s += G[(size_t)l * n + j] * x[l];
                }
                w[j] = c[j] - s;
            }
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += kT) xout[j] = x[j];
    if (threadIdx.x == 0) {
        out->iterations = it;
        out->converged = (s_status == 0 && it < max_iter) ? 1 : 0;
        out->status = s_status ? 2 : (it >= max_iter ? 1 : 0);
    }
}

constexpr int kSpgMemory = 10;        // nonmonotone line search: F compared with the max of the last 10
constexpr double kSpgGamma = 1e-4;    // sufficient-decrease constant of that test

// Gradient projection. bb = 0: Armijo's rule along the projection arc
// (Sec. 2.2.4), every trial step starting from s_bar = 1 / lambda_max(G).
// bb = 1: the spectral projected gradient of Birgin, Martinez & Raydan
// (2000): the step length before projection is Barzilai and Borwein's
// alpha = s's / s'y for the last move s and gradient change y, which on
// F = x'Gx - 2c'x + const is d'd / (2 d'Gd) whatever the fraction t of d
// taken; along d = P(x - alpha g) - x the full step is kept when F(x + t d)
// <= max(last kSpgMemory values of F) + gamma t g'd, else t becomes the
// minimiser of the quadratic through F(x), its slope and F(x + t d) (kept
// within [0.1 t, 0.9 t], t / 2 outside). F is quadratic along d, F(x + t d) =
// F + t g'd + t^2 d'Gd, so a trial costs no product with G. Both stop when
// the relative change of F falls below delta.
__global__ void __launch_bounds__(kT) k_projected_gradient(const double *__restrict__ G,
                                                           const double *__restrict__ cg, int n, double F0,
                                                           double delta, int max_iter, double sigma,
                                                           double beta, int bb, double *__restrict__ xio,
                                                           NnlsOut *out)
{
    extern __shared__ double sm[];
    double *x = sm, *gx = sm + n, *g = sm + 2 * n, *d = sm + 3 * n, *gd = sm + 4 * n, *v = sm + 5 * n;
    __shared__ double red[99];
    for (int j = threadIdx.x; j < n; j += kT) { x[j] = fmax(xio[j], 0.0); v[j] = rsqrt((double)n); }
    __syncthreads();
    // s_bar = 1 / lambda_max(G) by power iteration
    double lam = 0.0;
    for (int p = 0; p < 100; ++p) {
        for (int j = threadIdx.x; j < n; j += kT) {
            double s = 0.0;
            const double *gr = G + (size_t)j * n;
            for (int l = 0; l < n; ++l) s += gr[l] * v[l];
            gd[j] = s;
        }
        __syncthreads();
        double q = 0.0;
        for (int j = threadIdx.x; j < n; j += kT) q += gd[j] * gd[j];
        q = block_sum(q, red);
        const double nrm = sqrt(q);
        double rq = 0.0;
        for (int j = threadIdx.x; j < n; j += kT) rq += v[j] * gd[j];
        rq = block_sum(rq, red);
        lam = rq;
        for (int j = threadIdx.x; j < n; j += kT) v[j] = gd[j] / nrm;
        __syncthreads();
    }
    const double s_bar = 1.0 / lam;
    // G x
    for (int j = threadIdx.x; j < n; j += kT) {
        double s = 0.0;
        const double *gr = G + (size_t)j * n;
        for (int l = 0; l < n; ++l) s += gr[l] * x[l];
        gx[j] = s;
    }
    __syncthreads();
    double F = F0;
    int it = 0, conv = 0;
    double alpha = s_bar;
    // the last kSpgMemory values of F (every thread holds the same copy);
    // entries not yet written hold F0
    double hist[kSpgMemory];
    for (int k = 0; k < kSpgMemory; ++k) hist[k] = F0;
    while (bb && it < max_iter) {
        ++it;
        for (int j = threadIdx.x; j < n; j += kT) {
            g[j] = 2.0 * (gx[j] - cg[j]);
            d[j] = fmax(x[j] - alpha * g[j], 0.0) - x[j];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += kT) {
            double q = 0.0;
            const double *gr = G + (size_t)j * n;
            for (int l = 0; l < n; ++l) q += gr[l] * d[l];
            gd[j] = q;
        }
        __syncthreads();
        double gdot = 0.0, dgd = 0.0, dd = 0.0;
        for (int j = threadIdx.x; j < n; j += kT) { gdot += g[j] * d[j]; dgd += d[j] * gd[j]; dd += d[j] * d[j]; }
        block_sum3(gdot, dgd, dd, red);
        if (dd == 0.0 || gdot >= 0.0) { conv = 1; break; }       // P(x - alpha g) = x: x is stationary
        double Fref = F;
        for (int k = 0; k < kSpgMemory; ++k) Fref = fmax(Fref, hist[k]);
        double t = 1.0, dF = gdot + dgd;
        for (int trial = 0; trial < 200; ++trial) {
            dF = t * gdot + t * t * dgd;                          // F(x + t d) - F(x)
            if (F + dF <= Fref + kSpgGamma * t * gdot || t < 1e-30) break;
            const double tq = -0.5 * t * t * gdot / (dF - t * gdot);
            t = (tq >= 0.1 * t && tq <= 0.9 * t) ? tq : 0.5 * t;
        }
        for (int j = threadIdx.x; j < n; j += kT) { x[j] += t * d[j]; gx[j] += t * gd[j]; }
        __syncthreads();
        const double Fprev = F;
        F = F + dF;
        hist[it % kSpgMemory] = F;
        alpha = dgd > 0.0 ? fmin(fmax(dd / (2.0 * dgd), 1e-12 * s_bar), 1e12 * s_bar) : 1e12 * s_bar;
        if (fabs(dF) <= delta * fmax(Fprev, 1e-300)) { conv = 1; break; }
    }
    while (!bb && it < max_iter) {
        ++it;
        for (int j = threadIdx.x; j < n; j += kT) g[j] = 2.0 * (gx[j] - cg[j]);
        __syncthreads();
        double s = s_bar, dF = 0.0;
        for (int trial = 0; trial < 200; ++trial) {
            for (int j = threadIdx.x; j < n; j += kT) d[j] = fmax(x[j] - s * g[j], 0.0) - x[j];
            __syncthreads();
            for (int j = threadIdx.x; j < n; j += kT) {
                double q = 0.0;
                const double *gr = G + (size_t)j * n;
                for (int l = 0; l < n; ++l) q += gr[l] * d[l];
                gd[j] = q;
            }
            __syncthreads();
            double gdot = 0.0, dgd = 0.0;
            for (int j = threadIdx.x; j < n; j += kT) { gdot += g[j] * d[j]; dgd += d[j] * gd[j]; }
            double unused = 0.0;
            block_sum3(gdot, dgd, unused, red);
            dF = gdot + dgd;                      // F(x + d) - F(x)
            if (dF <= sigma * gdot || s < 1e-30) break;
            s *= beta;
        }
        for (int j = threadIdx.x; j < n; j += kT) { x[j] += d[j]; gx[j] += gd[j]; }
        __syncthreads();
        const double Fprev = F;
        F = F + dF;
        if (fabs(dF) <= delta * fmax(Fprev, 1e-300)) { conv = 1; break; }
    }
    for (int j = threadIdx.x; j < n; j += kT) xio[j] = x[j];
    if (threadIdx.x == 0) {
        out->iterations = it;
        out->converged = conv;
        out->status = conv ? 0 : 1;
        out->objective = F;
    }
}

// F(x) = ||A x - b||^2 and the KKT violation of x, after a solve
__global__ void __launch_bounds__(kT) k_nnls_report(const double *__restrict__ A, const double *__restrict__ b,
                                                    const double *__restrict__ G, const double *__restrict__ c,
                                                    const double *__restrict__ x, int m, int n, NnlsOut *out,
                                                    double *__restrict__ kkt)
{
    __shared__ double red[33];
    double f = 0.0;
    for (int r = threadIdx.x; r < m; r += kT) {
        double s = -b[r];
        const double *ar = A + (size_t)r * n;
        for (int l = 0; l < n; ++l) s += ar[l] * x[l];
        f += s * s;
    }
    f = block_sum(f, red);
    double viol = 0.0;
    for (int j = threadIdx.x; j < n; j += kT) {
        double s = 0.0;
        const double *gr = G + (size_t)j * n;
        for (int l = 0; l < n; ++l) s += gr[l] * x[l];
        const double gj = 2.0 * (s - c[j]);
        viol = fmax(viol, fmax(fmax(-x[j], -gj), fabs(x[j] * gj)));
    }
    for (int o = 16; o > 0; o >>= 1) viol = fmax(viol, __shfl_xor_sync(0xffffffffu, viol, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = viol;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < 32; ++w) v = fmax(v, red[w]);
        *kkt = v;
        out->objective = f;
    }
}

// The active-set kernel for n unknowns: the factor goes to shared memory
// when its packed lower triangle fits beside the other arrays.
cudaError_t launch_lawson_hanson(const double *G, const double *c, int n, double tol_scale, int max_iter, double *L,
                                 double *x, NnlsOut *out, cudaStream_t st)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t base = (size_t)n * 8 * 8, packed = base + (size_t)n * (n + 1) / 2 * 8;
    if (packed + 1024 <= (size_t)optin) {
        e = cudaFuncSetAttribute(k_lawson_hanson<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)packed);
        if (e != cudaSuccess) return e;
        k_lawson_hanson<true><<<1, kT, packed, st>>>(G, c, n, tol_scale, max_iter, L, x, out);
    } else {
        e = cudaFuncSetAttribute(k_lawson_hanson<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base);
        if (e != cudaSuccess) return e;
        k_lawson_hanson<false><<<1, kT, base, st>>>(G, c, n, tol_scale, max_iter, L, x, out);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace

lsm_status commission(const double *A, int32_t m, int32_t n, const double *b, lsm_mem mem,
                      const lsm_nnls_opts *opts, double *x, lsm_nnls_report *rep, cudaStream_t st)
{
    if (!A || !b || !x || m < 1 || n < 1 || n > 1024) return set_arg_error("lsm_commission: need m >= 1, 1 <= n <= 1024");
    lsm_nnls_opts o = {0, 0, 1e-12, 1e-4, 0.5, 0};
    if (opts) o = *opts;
    if (o.method < 0 || o.method > 2) return set_arg_error("lsm_commission: method must be 0, 1 or 2");
    if (o.max_iter <= 0) o.max_iter = o.method == 0 ? 3 * n : 200000;
    if (!(o.delta > 0)) o.delta = 1e-12;
    if (!(o.armijo_sigma > 0 && o.armijo_sigma < 1)) o.armijo_sigma = 1e-4;
    if (!(o.armijo_beta > 0 && o.armijo_beta < 1)) o.armijo_beta = 0.5;
    const size_t szA = (size_t)m * n * 8;
    char *buf = nullptr;
    const size_t need = (mem == LSM_MEM_HOST ? szA + (size_t)m * 8 : 0) + (size_t)n * n * 8 * 2 + (size_t)n * 8 * 2 +
                        64 + sizeof(NnlsOut) + 64;
    LSM_CUDA(cudaMalloc(&buf, need));
    const double *dA = A, *db = b;
    char *p = buf;
    if (mem == LSM_MEM_HOST) {
        double *tA = (double *)p; p += szA;
        double *tb = (double *)p; p += (size_t)m * 8;
        cudaError_t e1 = cudaMemcpyAsync(tA, A, szA, cudaMemcpyHostToDevice, st);
        cudaError_t e2 = cudaMemcpyAsync(tb, b, (size_t)m * 8, cudaMemcpyHostToDevice, st);
        if (e1 != cudaSuccess || e2 != cudaSuccess) { cudaFree(buf); return set_cuda_error(e1 ? e1 : e2, "copy A,b"); }
        dA = tA; db = tb;
    }
    double *G = (double *)p; p += (size_t)n * n * 8;
    double *L = (double *)p; p += (size_t)n * n * 8;
    double *c = (double *)p; p += (size_t)n * 8;
    double *dx = (double *)p; p += (size_t)n * 8;
    double *kkt = (double *)p; p += 64;
    NnlsOut *dout = (NnlsOut *)p;
    lsm_status rc = LSM_OK;
    cudaError_t e = cudaSuccess;
    NnlsOut hout = {0, 0, 0, 0.0};
    double hkkt = 0.0;
    do {
        dim3 gb((n + 31) / 32, (n + 31) / 32);
        k_gram<<<gb, dim3(32, 8), 0, st>>>(dA, db, m, n, G, c);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if (o.method == 0) {
            const double tol_scale = 10.0 * 2.220446049250313e-16 * (m > n ? m : n);
            if ((e = launch_lawson_hanson(G, c, n, tol_scale, o.max_iter, L, dx, dout, st)) != cudaSuccess) break;
        } else {
            // starting point: x (use_x0) or all ones (the uncommissioned weights)
            std::vector<double> x0((size_t)n, 1.0);
            if (o.use_x0) for (int j = 0; j < n; ++j) x0[j] = x[j];
            if ((e = cudaMemcpyAsync(dx, x0.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
            k_nnls_report<<<1, kT, 0, st>>>(dA, db, G, c, dx, m, n, dout, kkt);
            count_launch();
            NnlsOut f0;
            if ((e = cudaMemcpyAsync(&f0, dout, sizeof(NnlsOut), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
            const size_t smem = (size_t)n * 8 * 6;
            cudaFuncSetAttribute(k_projected_gradient, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_projected_gradient<<<1, kT, smem, st>>>(G, c, n, f0.objective, o.delta, o.max_iter, o.armijo_sigma,
                                                      o.armijo_beta, o.method == 2, dx, dout);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) break;
        }
        NnlsOut keep;
        if ((e = cudaMemcpyAsync(&keep, dout, sizeof(NnlsOut), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        k_nnls_report<<<1, kT, 0, st>>>(dA, db, G, c, dx, m, n, dout, kkt);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&hout, dout, sizeof(NnlsOut), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&hkkt, kkt, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(x, dx, (size_t)n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        hout.iterations = keep.iterations;
        hout.converged = keep.converged;
        hout.status = keep.status;
    } while (0);
    cudaFree(buf);
    if (e != cudaSuccess) return set_cuda_error(e, "lsm_commission");
    if (rep) {
        rep->iterations = hout.iterations;
        rep->converged = hout.converged;
        rep->objective = hout.objective;
        rep->kkt = hkkt;
    }
    if (hout.status == 2) return set_arg_error("lsm_commission: passive-set Gram matrix not positive definite");
    if (hout.status == 1) rc = LSM_ERR_NOT_CONVERGED;
    return rc;
}


// ---------------------------------------------------------------------------
// Allocation-free variant (lsm_commission_static).
//
// Some callers may not allocate GPU memory while they run: a planning service
// that reserves all of its device memory up front and forbids growth during a
// session, or a host application that owns the GPU memory and embeds this
// library as a plugin. For them the solve's scratch (the Gram matrix, its
// Cholesky factor, A^T b and the small result records) lives in one fixed
// device array that the library holds from load until process exit. Its size
// caps the number of unknowns at kStaticMaxN.
namespace {

constexpr int kStaticMaxN = 256;
constexpr size_t kStaticGram = (size_t)kStaticMaxN * kStaticMaxN;
// G, L (n x n each, packed with stride n), c (n), KKT value (8), result record (8)
constexpr size_t kStaticDoubles = 2 * kStaticGram + kStaticMaxN + 16;

static __device__ __align__(256) double g_nnls_scratch[kStaticDoubles];

// Device address of g_nnls_scratch per device, looked up once per device on
// the first call with that device current. The cache assumes one CUDA context
// per device for the life of the process (the runtime's primary context): after
// cudaDeviceReset the module may be loaded again at another address, so a
// process that resets a device must not call lsm_commission_static afterwards.
std::mutex g_scratch_mu;
double *g_scratch_ptr[64] = {};

__global__ void k_fill(double *__restrict__ x, double v, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// A, b and x must be memory the GPU addresses directly (device or managed
// allocations). cudaPointerGetAttributes allocates nothing; a host pointer
// would otherwise reach the kernels and fault.
lsm_status check_device_pointer(const void *p, const char *what)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_arg_error((std::string("lsm_commission_static: ") + what + " is not a device pointer").c_str());
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_arg_error((std::string("lsm_commission_static: ") + what +
                              " must be device or managed memory (got host or unregistered memory)").c_str());
    return LSM_OK;
}

lsm_status scratch_address(double **out)
{
    int dev = 0;
    LSM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_arg_error("lsm_commission_static: device index above 63");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_nnls_scratch);
        if (e != cudaSuccess) return set_cuda_error(e, "lsm_commission_static: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LSM_OK;
}

}  // namespace

}  // namespace lsm

extern "C" lsm_status lsm_commission_static(const double *A, int32_t m, int32_t n, const double *b,
                                            const lsm_nnls_opts *opts, double *x, lsm_nnls_report *report,
                                            lsm_stream stream)
{
    using namespace lsm;
    cudaStream_t st = (cudaStream_t)stream;
    if (!A || !b || !x || m < 1 || n < 1) return set_arg_error("lsm_commission_static: NULL pointer or empty problem");
    if (n > kStaticMaxN)
        return set_arg_error("lsm_commission_static: at most 256 unknowns fit the fixed scratch; use lsm_commission");
    if (lsm_status pc = check_device_pointer(A, "A")) return pc;
    if (lsm_status pc = check_device_pointer(b, "b")) return pc;
    if (lsm_status pc = check_device_pointer(x, "x")) return pc;
    lsm_nnls_opts o = {0, 0, 1e-12, 1e-4, 0.5, 0};
    if (opts) o = *opts;
    if (o.method < 0 || o.method > 2) return set_arg_error("lsm_commission_static: method must be 0, 1 or 2");
    if (o.max_iter <= 0) o.max_iter = o.method == 0 ? 3 * n : 200000;
    if (!(o.delta > 0)) o.delta = 1e-12;
    if (!(o.armijo_sigma > 0 && o.armijo_sigma < 1)) o.armijo_sigma = 1e-4;
    if (!(o.armijo_beta > 0 && o.armijo_beta < 1)) o.armijo_beta = 0.5;
    double *base = nullptr;
    lsm_status rc = scratch_address(&base);
    if (rc) return rc;
    double *G = base, *L = base + kStaticGram, *c = base + 2 * kStaticGram;
    double *kkt = c + kStaticMaxN;
    NnlsOut *dout = (NnlsOut *)(kkt + 8);
    // the array keeps the previous call's contents: reset the result record
    LSM_CUDA(cudaMemsetAsync(dout, 0, sizeof(NnlsOut), st));
    LSM_CUDA(cudaMemsetAsync(kkt, 0, 8, st));
    dim3 gb((n + 31) / 32, (n + 31) / 32);
    k_gram<<<gb, dim3(32, 8), 0, st>>>(A, b, m, n, G, c);
    LSM_LAUNCHED("k_gram");
    if (o.method == 0) {
        const double tol_scale = 10.0 * 2.220446049250313e-16 * (m > n ? m : n);
        LSM_CUDA(launch_lawson_hanson(G, c, n, tol_scale, o.max_iter, L, x, dout, st));
    } else {
        if (!o.use_x0) {
            k_fill<<<(n + 255) / 256, 256, 0, st>>>(x, 1.0, n);
            LSM_LAUNCHED("k_fill");
        }
        k_nnls_report<<<1, kT, 0, st>>>(A, b, G, c, x, m, n, dout, kkt);
        LSM_LAUNCHED("k_nnls_report");
        NnlsOut f0;
        LSM_CUDA(cudaMemcpyAsync(&f0, dout, sizeof(NnlsOut), cudaMemcpyDeviceToHost, st));
        LSM_CUDA(cudaStreamSynchronize(st));
        const size_t smem = (size_t)n * 8 * 6;
        LSM_CUDA(cudaFuncSetAttribute(k_projected_gradient, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_projected_gradient<<<1, kT, smem, st>>>(G, c, n, f0.objective, o.delta, o.max_iter, o.armijo_sigma,
                                                  o.armijo_beta, o.method == 2, x, dout);
        LSM_LAUNCHED("k_projected_gradient");
    }
    NnlsOut keep, fin;
    LSM_CUDA(cudaMemcpyAsync(&keep, dout, sizeof(NnlsOut), cudaMemcpyDeviceToHost, st));
    k_nnls_report<<<1, kT, 0, st>>>(A, b, G, c, x, m, n, dout, kkt);
    LSM_LAUNCHED("k_nnls_report");
    double hk = 0.0;
    LSM_CUDA(cudaMemcpyAsync(&fin, dout, sizeof(NnlsOut), cudaMemcpyDeviceToHost, st));
    LSM_CUDA(cudaMemcpyAsync(&hk, kkt, 8, cudaMemcpyDeviceToHost, st));
    LSM_CUDA(cudaStreamSynchronize(st));
    if (report) {
        report->iterations = keep.iterations;
        report->converged = keep.converged;
        report->objective = fin.objective;
        report->kkt = hk;
    }
    if (keep.status == 2) return set_arg_error("lsm_commission_static: passive-set Gram matrix not positive definite");
    return keep.status == 1 ? LSM_ERR_NOT_CONVERGED : LSM_OK;
}

