// sample.cuh -- on-the-fly source sampling, steps S3-S5 (Eq. 4-7).
#pragma once

#include "handles.cuh"

namespace lsm {

struct SrcParticle {
    float x, y, u, v, w, E;   // position on the phantom-surface plane, direction, energy
    float xp, yp;             // position on the phase-space plane
    int stype, ebin, ring, comp, psr, beam;
    int64_t entry;
    bool accepted;
};

// largest entry k with start[k] <= h
__device__ __forceinline__ int64_t find_entry(const int64_t *__restrict__ start, int64_t n_ent, int64_t h)
{
    int64_t lo = 0, hi = n_ent - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= h) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void lanemask_lt(unsigned &m) { asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m)); }

// The same search for a warp whose lanes hold plan positions (valid lanes
// first): when they are consecutive, one 32-way search finds the first lane's
// entry and every lane walks forward from it (a warp spans a few entries);
// otherwise each lane searches alone. All 32 lanes must call it.
__device__ __forceinline__ int64_t find_entry_warp(const int64_t *__restrict__ start, int64_t n_ent, int64_t h,
                                                   bool valid)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    if (vm == 0u) return 0;
    const int nv = __popc(vm);
    const int64_t h0 = __shfl_sync(0xffffffffu, h, 0);
    const int64_t hl = __shfl_sync(0xffffffffu, h, nv - 1);
    if ((vm & 1u) == 0u || hl - h0 != (int64_t)(nv - 1)) return valid ? find_entry(start, n_ent, h) : 0;
    int64_t lo = 0, hi = n_ent - 1;            // start[lo] <= h0 < start[hi + 1]
    while (hi - lo >= 32) {
        const int64_t step = (hi - lo + 32) / 32;
        const int64_t piv = lo + (int64_t)lane * step;
        const bool le = piv <= hi && __ldg(start + piv) <= h0;
        const unsigned b = __ballot_sync(0xffffffffu, le);
        const int top = 31 - __clz(b);          // lane 0's pivot is lo, always <= h0
        lo = lo + (int64_t)top * step;
        const int64_t nh = lo + step - 1;
        hi = nh < hi ? nh : hi;
    }
    {
        const int64_t piv = lo + lane;
        const bool le = piv <= hi && __ldg(start + piv) <= h0;
        lo += 31 - __clz(__ballot_sync(0xffffffffu, le));
    }
    int64_t k = lo;
    if (valid)
        for (int it = 0; it < 32 && k + 1 < n_ent && __ldg(start + k + 1) <= h; ++it) ++k;
    return k;
}

// One history: plan position h of history g; z_rel = phantom surface - z_phsp.
__device__ __forceinline__ void sample_history(const SampleParams &P, uint32_t k0, uint32_t k1, uint64_t g,
                                               int64_t h, float z_rel, SrcParticle &o, int64_t k = -1)
{
    if (k < 0) k = find_entry(P.start, __ldg(P.n_ent), h);
    const EntryRec en = P.ent[k];
    const uint32_t glo = (uint32_t)g, ghi = (uint32_t)(g >> 32);
    const uint4 a = philox4x32_10(k0, k1, glo, ghi, 0u, 0u);
    const uint4 b = philox4x32_10(k0, k1, glo, ghi, 0u, 1u);

    // position uniform in the PSL and energy uniform in the bin (S3); the
    // position is formed without FMA so that the ring decision below is the
    // one any single-precision evaluation of these two operations gives
    const float pf = P.pitch;
    const float x = __fadd_rn(__fmul_rn((float)((int)en.ix - P.n_r), pf), __fmul_rn(u01(a.x), pf));
    const float y = __fadd_rn(__fmul_rn((float)((int)en.iy - P.n_r), pf), __fmul_rn(u01(a.y), pf));
    const int s = en.stype, e = en.ebin;
    const float E = P.e_lo[s] + ((float)e + u01(a.z)) * P.de[s];

    // ring that holds the sampled radius (S4): the largest kk < n_r with
    // r2 >= (kk pf)^2, both products rounded as written. The test is monotone
    // in kk, so an estimate from r / pf is corrected by single steps until it
    // is the largest kk passing (the estimate only saves steps)
    const float r2 = __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
    auto inside = [&](int kk) {
        const float ek = __fmul_rn((float)kk, pf);
        return r2 >= __fmul_rn(ek, ek);
    };
    int ring = r2 > 0.0f ? (int)__fdividef(r2 * rsqrtf(r2), pf) : 0;
    ring = min(max(ring, 0), P.n_r - 1);
    while (ring + 1 < P.n_r && inside(ring + 1)) ++ring;
    while (ring > 0 && !inside(ring)) --ring;

    // Box-Muller pair
    const float rad = sqrtf(-2.0f * __logf(u01(b.x)));
    float sn, cs;
    sincospif(2.0f * u01(b.y), &sn, &cs);
    const float n1 = rad * cs, n2 = rad * sn;

    // PSR index carried for the basis tally
    const int R = en.fixed_ring >= 0 ? en.fixed_ring : (b.z < en.thr ? (int)en.r0 : (int)en.r0 + 1);

    // radius and its reciprocal from one reciprocal square root
    const float rinv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    const float r = r2 * rinv;
    float u0, v0, w0;
    int comp = -1;
    if (s == 0) {
        // Eq. 4-5: Gaussian focal spot, direction to (r, 0, z_phsp) in the local frame
        const float xs = P.sigma_s * n1, ys = P.sigma_s * n2;
        const float dxs = r - xs;
        const float inv = rsqrtf(dxs * dxs + ys * ys + P.z_phsp * P.z_phsp);
        u0 = dxs * inv; v0 = -ys * inv; w0 = P.z_phsp * inv;
    } else {
        const int pi = e * P.n_r + ring;
        float al, be;
        if (s == 1) {
            // Eq. 6: component by the cumulative table, then the Gaussian pair
            const unsigned long long t1 = P.mixthr[2 * pi], t2 = P.mixthr[2 * pi + 1];
            comp = ((unsigned long long)a.w < t1) ? 0 : (((unsigned long long)a.w < t2) ? 1 : 2);
            const float4 m = P.mix[3 * pi + comp];
            al = m.x + m.y * n1;
            be = m.z * n2;
        } else {
            const float2 es = P.esig[pi];            // Eq. 7
            al = es.x * n1;
            be = es.y * n2;
        }
        const float ta = tanf(al), tb = tanf(be);    // alpha = atan(u/w), beta = atan(v/w)
        const float inv = rsqrtf(ta * ta + tb * tb + 1.0f);
        u0 = ta * inv; v0 = tb * inv; w0 = inv;
    }
    // rotate the local frame (u along the radius) by the polar angle of (x, y)
    float c = 1.0f, sv = 0.0f;
    if (r2 > 0.0f) { c = x * rinv; sv = y * rinv; }
    const float u = u0 * c - v0 * sv, v = u0 * sv + v0 * c, w = w0;

    // jaw rejection at the upper jaw surfaces, straight flight to the phantom
    const float *J = P.jaws_f + 4 * en.beam;
    const float iw = 1.0f / w;
    const float yJ = y + P.zy_rel * v * iw, xJ = x + P.zx_rel * u * iw;
    o.accepted = yJ >= J[0] && yJ <= J[1] && xJ >= J[2] && xJ <= J[3];
    o.x = x + z_rel * u * iw;
    o.y = y + z_rel * v * iw;
    o.u = u; o.v = v; o.w = w; o.E = E;
    o.xp = x; o.yp = y;
    o.stype = s; o.ebin = e; o.ring = ring; o.comp = comp;
    o.psr = (s * P.n_e + e) * P.n_r + R;
    o.beam = en.beam;
    o.entry = k;
}

}  // namespace lsm
