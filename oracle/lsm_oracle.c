/*
 * lsm_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, single-threaded FP64 restatement of the analytic linac source
 * model in use, after Tian et al., "An analytic linear accelerator source model
 * for Monte Carlo dose calculations. II" (arXiv:1503.01725):
 *
 *   - PSR -> PSL weight conversion, Sec. 2.1.1, Eq. 1-2 and its four steps;
 *   - sampling areas for primary and scatter/electron sub-sources, Sec. 2.1.2
 *     and the Fig. 3 caption;
 *   - particles per PSL, Eq. 3 (step S2);
 *   - primary photon sampling, Eq. 4-5 (step S3); scatter photon sampling with
 *     the K=3 Gaussian mixture, Eq. 6 and its cumulative table (step S4);
 *     electron sampling, Eq. 7 (step S5); rotation by the polar angle of (x,y)
 *     and jaw rejection at the upper jaw surfaces;
 *   - the loop order of Sec. 2.1.3 (sub-source, energy bin outer, PSL inner);
 *   - the PSR-indexed basis-dose tally of Sec. 2.2.2 (3D index array, 2D dose
 *     array [row][PSR], secondaries inherit the PSR index);
 *   - multi-beam plans (step S1 loops over beams; the prostate and H&N cases of
 *     Table 1): each beam turned by its gantry angle about the isocentre, the
 *     particle entering the phantom where its straight line meets the voxel box
 *     (the geometry is the textbook rotation and slab test; the paper gives no
 *     formula).
 *
 * The paper does not describe its transport physics (Sec. 2.3 gives only the
 * 200 keV electron and 50 keV photon cutoffs). This file therefore implements
 * the stated simplification: photons by Woodcock tracking with Compton
 * (Klein-Nishina, sampled by inverting its closed-form CDF), photoelectric and pair
 * interactions whose cross sections come from closed forms with two synthetic
 * constants; electrons by condensed-history CSDA steps with Bethe collision
 * stopping power and a Gaussian (Highland) multiple-scattering deflection.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
 * from that paper's definition. Key = (seed_lo, seed_hi); counter =
 * (history_lo, history_hi, stream id, draw index). u32 -> (0,1] by
 * ((x >> 8) + 1) * 2^-24.
 *
 * Nothing in the product imports, links or runs this file; only the tests, the
 * smoke check and the benchmark's CPU baseline do. It shares no code with the
 * CUDA path.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liblsm_oracle.so
 * (no FMA contraction, so FP64 results of +,-,*,/,sqrt are the IEEE ones).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------- */

OR_API void or_philox4x32_10(const uint32_t key_in[2], const uint32_t ctr_in[4],
                             uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;           /* Weyl sequence bump of the key */
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u01(uint32_t x) { return ((double)(x >> 8) + 1.0) * (1.0 / 16777216.0); }
static float u01f(uint32_t x) { return ((float)(x >> 8) + 1.0f) * (1.0f / 16777216.0f); }

typedef struct {
    uint32_t key[2];
    uint32_t g_lo, g_hi, sid, ctr;
} stream_t;

static void stream_init(stream_t *s, uint64_t seed, uint64_t g, uint32_t sid)
{
    s->key[0] = (uint32_t)seed; s->key[1] = (uint32_t)(seed >> 32);
    s->g_lo = (uint32_t)g; s->g_hi = (uint32_t)(g >> 32);
    s->sid = sid; s->ctr = 0;
}

static void draw(stream_t *s, uint32_t out[4])
{
    uint32_t c[4] = {s->g_lo, s->g_hi, s->sid, s->ctr};
    or_philox4x32_10(s->key, c, out);
    s->ctr++;
}

/* MurmurHash3's 32-bit finaliser (Appleby). */
static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* Stream id of the slot-th particle created at one interaction: a hash of the
 * parent's stream id and its current draw counter. Ids 0 (source sampling) and
 * 1 (primary transport) are reserved. */
static uint32_t child_id(const stream_t *s, uint32_t slot)
{
    uint32_t h = fmix32(s->sid ^ fmix32(s->ctr ^ (0x9E3779B9u * (slot + 1u))));
    return h < 2u ? h + 2u : h;
}

/* ------------------------------------------------------------------------- */
/* Interaction data: closed forms (stated synthetic transport model)          */
/* ------------------------------------------------------------------------- */

#define ME 0.51099895             /* electron rest energy, MeV */
#define RE 2.8179403262e-13       /* classical electron radius, cm */
#define PI_D 3.14159265358979323846
#define E_CUT_E 0.2               /* electron transport cutoff, MeV (Sec. 2.3) */
#define E_CUT_G 0.05              /* photon transport cutoff, MeV (Sec. 2.3) */

/* material classes: 0 water-like (air, lung, soft tissue, water), 1 bone */
static const double NE_G[2] = {3.34e23, 3.34e23 * 0.96};  /* electrons / g */
static const double ZEFF[2] = {7.4, 13.8};
static const double IEV[2] = {75.0, 106.4};                /* mean excitation, eV */
static const double X0G[2] = {36.08, 21.68};               /* radiation length, g/cm2 */

/* Klein-Nishina total cross section per electron, cm^2 (closed form). */
OR_API double or_kn_sigma(double E)
{
    double k = E / ME, a = 1.0 + 2.0 * k, L = log(a);
    return 2.0 * PI_D * RE * RE *
           ((1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k) + L / (2.0 * k) -
            (1.0 + 3.0 * k) / (a * a));
}

/* Photoelectric: C_pe Z^3 / E^3 per electron, C_pe fixed by
 * mu_pe = mu_compton at 30 keV in water (Z = 7.4). */
static double c_pe(void) { return or_kn_sigma(0.03) * 0.03 * 0.03 * 0.03 / (7.4 * 7.4 * 7.4); }
static double sigma_pe(double E, double Z) { return c_pe() * Z * Z * Z / (E * E * E); }

/* Pair: C_pp Z (E - 2mc^2)/E per electron above threshold, C_pp fixed by
 * mu_pair / mu_total = 0.05 at 6 MeV in water. */
static double c_pp(void)
{
    double s = (0.05 / 0.95) * (or_kn_sigma(6.0) + sigma_pe(6.0, 7.4));
    return s * 6.0 / (7.4 * (6.0 - 2.0 * ME));
}
static double sigma_pp(double E, double Z) { return E > 2.0 * ME ? c_pp() * Z * (E - 2.0 * ME) / E : 0.0; }

/* Mass attenuation coefficients (cm^2/g); comp 0 Compton, 1 photo, 2 pair, 3 total. */
OR_API double or_mu_mass(double E, int m, int comp)
{
    double c = NE_G[m] * or_kn_sigma(E);
    double p = NE_G[m] * sigma_pe(E, ZEFF[m]);
    double q = NE_G[m] * sigma_pp(E, ZEFF[m]);
    switch (comp) {
    case 0: return c;
    case 1: return p;
    case 2: return q;
    default: return c + p + q;
    }
}

/* Bethe collision stopping power for electrons (no density effect), MeV cm^2/g. */
OR_API double or_scol_mass(double E, int m)
{
    double tau = E / ME, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double im = IEV[m] * 1e-6 / ME;
    double F = 1.0 - b2 + (tau * tau / 8.0 - (2.0 * tau + 1.0) * log(2.0)) / (g * g);
    double brk = log(tau * tau * (tau + 2.0) / (2.0 * im * im)) + F;
    return 2.0 * PI_D * RE * RE * ME * NE_G[m] / b2 * brk;
}

/* Highland multiple-scattering width (rad) for kinetic energy E over t radiation lengths. */
OR_API double or_highland(double E, double t)
{
    double bcp = E * (E + 2.0 * ME) / (E + ME);
    double f = 1.0 + 0.038 * log(t);
    if (f < 0.0) f = 0.0;
    return 13.6 / bcp * sqrt(t) * f;
}

/* ------------------------------------------------------------------------- */
/* Model, beams, plan                                                         */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n_e, n_r;
    double dr, z_phsp, sigma_s;
    double e_lo[3], de[3];
    const double *w;                       /* [3][n_e][n_r] PSR weights */
    const double *mix_c, *mix_mu, *mix_sa, *mix_sb; /* [n_e][n_r][3] */
    const double *e_sa, *e_sb;             /* [n_e][n_r] */
} or_model;

typedef struct {
    double sad, z_jaw_y, z_jaw_x;  /* upper surfaces of the Y and X jaws */
    int32_t n_beams;
    const double *jaws;            /* [n_beams][4]: x1 x2 y1 y2 at the isocentre plane */
    const double *gantry;          /* NULL, or [n_beams] gantry angles (radians) */
    double iso[3];                 /* isocentre in phantom coordinates (with gantry) */
} or_beams;

typedef struct {
    int n_e, n_r, n_xy, n_beams;
    double p;                      /* PSL pitch */
    or_model M;                    /* pointers borrowed for the plan's lifetime */
    double sad, z_jaw_y, z_jaw_x;
    double *jaws;                  /* copy [n_beams][4] */
    int rotated;                   /* gantry angles given */
    double gantry[16], iso[3];
    double *wpsl;                  /* [3][n_e][n_xy][n_xy] normalised PSL weight */
    int32_t *tag_r0;               /* [n_xy][n_xy] lower ring of the interpolation */
    double *tag_l0;                /* [n_xy][n_xy] lambda of the lower ring */
    double *area;                  /* [n_beams][2][4] xa xb ya yb; class 0 primary, 1 scatter+electron */
    uint8_t *incl;                 /* [n_beams][2][n_xy][n_xy] */
    double denom;                  /* Eq. 3 denominator (whole-plan mode) */
    int64_t n_hist;                /* histories of one pass over the plan */
    int64_t *count;                /* whole-plan mode: [n_beams][3][n_e][n_xy][n_xy] */
    /* plan entries in loop order (non-zero counts only) */
    int64_t n_ent;
    int64_t *ent_start;            /* exclusive prefix */
    int32_t *ent_b, *ent_s, *ent_e, *ent_ix, *ent_iy, *ent_tag;  /* tag -1: drawn */
    double *ent_scale;             /* per-PSR mode: D_{k,b} / n_k ; whole-plan: 0 */
    int per_psr;
} or_plan;

/* Linear interpolation of the ring density W_R / dr in r (Sec. 2.1.1, step 2),
 * with ring values placed at ring centres; clamped to ring 0 inside the first
 * centre and to the last ring between the last centre and the outer edge; zero
 * beyond the outer edge. Returns the lower ring and its lambda. */
static void ring_interp(double r, int n_r, double dr, int *r0, double *l0, int *inside)
{
    *inside = 1;
    if (r >= (double)n_r * dr) { *r0 = n_r - 1; *l0 = 1.0; *inside = 0; return; }
    double t = r / dr - 0.5;
    if (t <= 0.0) { *r0 = 0; *l0 = 1.0; return; }
    if (t >= (double)(n_r - 1)) { *r0 = n_r - 1; *l0 = 1.0; return; }
    int i = (int)floor(t);
    *r0 = i; *l0 = 1.0 - (t - (double)i);
}

static int cmp_rem_desc(const void *a, const void *b);
typedef struct { double rem; int64_t idx; } remrec;
static int cmp_rem_desc(const void *a, const void *b)
{
    const remrec *x = (const remrec *)a, *y = (const remrec *)b;
    if (x->rem > y->rem) return -1;
    if (x->rem < y->rem) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* Largest-remainder rounding of q[0..n) (sum exactly `total`), ties to the
 * lower index. */
static void hamilton(const double *q, int64_t n, int64_t total, int64_t *out)
{
    int64_t s = 0;
    remrec *rr = (remrec *)malloc(sizeof(remrec) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) {
        double f = floor(q[j]);
        out[j] = (int64_t)f;
        s += out[j];
        rr[j].rem = q[j] - f; rr[j].idx = j;
    }
    int64_t left = total - s;
    qsort(rr, (size_t)n, sizeof(remrec), cmp_rem_desc);
    for (int64_t j = 0; j < left && j < n; ++j) out[rr[j].idx] += 1;
    free(rr);
}

/* Sampling areas on the phase-space plane (Sec. 2.1.2, Fig. 3). */
static void sampling_areas(const or_plan *P, int b, double out[2][4])
{
    const double *j = &P->jaws[4 * b];
    double x1 = j[0], x2 = j[1], y1 = j[2], y2 = j[3];
    double zp = P->M.z_phsp, sad = P->sad;
    /* primary: jaw opening scaled back to the plane */
    double k = zp / sad;
    out[0][0] = x1 * k; out[0][1] = x2 * k; out[0][2] = y1 * k; out[0][3] = y2 * k;
    /* scatter / electrons: back-project the upper jaw surfaces from the field
     * centre on the isocentre plane; X and Y jaws sit at different z */
    double cx = 0.5 * (x1 + x2), cy = 0.5 * (y1 + y2);
    double fx = (sad - zp) / (sad - P->z_jaw_x), fy = (sad - zp) / (sad - P->z_jaw_y);
    double kx = P->z_jaw_x / sad, ky = P->z_jaw_y / sad;
    out[1][0] = cx + (x1 * kx - cx) * fx;
    out[1][1] = cx + (x2 * kx - cx) * fx;
    out[1][2] = cy + (y1 * ky - cy) * fy;
    out[1][3] = cy + (y2 * ky - cy) * fy;
}

static void plan_free(or_plan *P)
{
    if (!P) return;
    free(P->jaws); free(P->wpsl); free(P->tag_r0); free(P->tag_l0); free(P->area);
    free(P->incl); free(P->count); free(P->ent_start); free(P->ent_b); free(P->ent_s);
    free(P->ent_e); free(P->ent_ix); free(P->ent_iy); free(P->ent_tag); free(P->ent_scale);
    free(P);
}

OR_API void or_plan_free(void *h) { plan_free((or_plan *)h); }

static void ent_alloc(or_plan *P, int64_t n)
{
    size_t m = (size_t)(n > 0 ? n : 1);
    P->ent_start = (int64_t *)calloc(m + 1, sizeof(int64_t));
    P->ent_b = (int32_t *)calloc(m, 4); P->ent_s = (int32_t *)calloc(m, 4);
    P->ent_e = (int32_t *)calloc(m, 4); P->ent_ix = (int32_t *)calloc(m, 4);
    P->ent_iy = (int32_t *)calloc(m, 4); P->ent_tag = (int32_t *)calloc(m, 4);
    P->ent_scale = (double *)calloc(m, 8);
}

/* The plan's sums over the PSLs of a block (step 4's raw total, Eq. 3's
 * partial denominators, a basis run's denominator) in one fixed order, so
 * that any implementation reproduces them bit for bit: 32 interleaved
 * partial sums, partial l adding x[l], x[l + 32], x[l + 64], ... in index
 * order from 0.0, then combined by halving, partial l += partial l + h for
 * h = 16, 8, 4, 2, 1; the result is partial 0. With a mask, excluded
 * elements contribute +0.0 (which leaves a sum of non-negative terms
 * unchanged). The paper fixes no order; a sequential sum of 400 FP64 terms
 * is a chain of 400 dependent adds, this one a chain of 18. */
OR_API double or_sum32(const double *x, const uint8_t *mask, int64_t n)
{
    double t[32];
    for (int l = 0; l < 32; ++l) {
        double a = 0.0;
        for (int64_t j = l; j < n; j += 32) a += (mask && !mask[j]) ? 0.0 : x[j];
        t[l] = a;
    }
    for (int h = 16; h >= 1; h >>= 1)
        for (int l = 0; l < h; ++l) t[l] = t[l] + t[l + h];
    return t[0];
}

/*
 * Build the PSL representation and the sampling plan.
 *   per_psr_n == NULL: whole-source plan, n_hist histories shared by Eq. 3 over
 *       all beams, sub-sources, energy bins and included PSLs.
 *   per_psr_n != NULL: one basis run per (PSR k, beam b) with per_psr_n[k]
 *       histories each, PSL weights restricted to PSR k's interpolation share
 *       (the k-th term of the linear map W_R -> W_XY); n_hist is ignored.
 */
OR_API void *or_plan_build(const or_model *M, const or_beams *B, int64_t n_hist,
                           const int64_t *per_psr_n)
{
    or_plan *P = (or_plan *)calloc(1, sizeof(or_plan));
    int ne = M->n_e, nr = M->n_r, nxy = 2 * nr, nb = B->n_beams;
    P->n_e = ne; P->n_r = nr; P->n_xy = nxy; P->n_beams = nb; P->p = M->dr; P->M = *M;
    P->sad = B->sad; P->z_jaw_y = B->z_jaw_y; P->z_jaw_x = B->z_jaw_x;
    P->jaws = (double *)malloc(sizeof(double) * 4 * (size_t)nb);
    memcpy(P->jaws, B->jaws, sizeof(double) * 4 * (size_t)nb);
    P->rotated = B->gantry != NULL;
    for (int b = 0; b < nb && b < 16; ++b) P->gantry[b] = B->gantry ? B->gantry[b] : 0.0;
    for (int k = 0; k < 3; ++k) P->iso[k] = B->gantry ? B->iso[k] : (k == 2 ? B->sad : 0.0);
    size_t npsl = (size_t)nxy * nxy;
    P->wpsl = (double *)calloc(3 * (size_t)ne * npsl, sizeof(double));
    P->tag_r0 = (int32_t *)calloc(npsl, 4);
    P->tag_l0 = (double *)calloc(npsl, 8);
    P->area = (double *)calloc((size_t)nb * 8, 8);
    P->incl = (uint8_t *)calloc((size_t)nb * 2 * npsl, 1);
    double p = M->dr;

    /* Sec. 2.1.1 steps 1-3 per PSL centre; step 4 per (sub-source, energy) block */
    for (int s = 0; s < 3; ++s)
        for (int e = 0; e < ne; ++e) {
            const double *W = &M->w[((size_t)s * ne + e) * nr];
            double *out = &P->wpsl[((size_t)s * ne + e) * npsl];
            double sraw = 0.0;
            for (int iy = 0; iy < nxy; ++iy)
                for (int ix = 0; ix < nxy; ++ix) {
                    double xc = ((double)(ix - nr) + 0.5) * p;
                    double yc = ((double)(iy - nr) + 0.5) * p;
                    double r = sqrt(xc * xc + yc * yc);            /* step 1 */
                    int r0, in; double l0;
                    ring_interp(r, nr, M->dr, &r0, &l0, &in);
                    double dens = 0.0;                              /* step 2 */
                    if (in) {
                        dens = l0 * (W[r0] / M->dr);
                        if (l0 < 1.0) dens += (1.0 - l0) * (W[r0 + 1] / M->dr);
                    }
                    double raw = dens / (2.0 * PI_D * r);           /* step 3 */
                    out[iy * nxy + ix] = raw;
                    if (s == 0 && e == 0) {
                        P->tag_r0[iy * nxy + ix] = r0;
                        P->tag_l0[iy * nxy + ix] = in ? l0 : 0.0;
                    }
                }
            sraw = or_sum32(out, NULL, (int64_t)npsl);
            double sR = 0.0;
            for (int R = 0; R < nr; ++R) sR += W[R];
            double scale = sraw > 0.0 ? sR / sraw : 0.0;           /* step 4 */
            for (size_t j = 0; j < npsl; ++j) out[j] = out[j] * scale;
        }

    /* sampling areas and PSL inclusion (positive-area overlap) */
    for (int b = 0; b < nb; ++b) {
        double ar[2][4];
        sampling_areas(P, b, ar);
        for (int c = 0; c < 2; ++c) {
            for (int q = 0; q < 4; ++q) P->area[(b * 2 + c) * 4 + q] = ar[c][q];
            for (int iy = 0; iy < nxy; ++iy)
                for (int ix = 0; ix < nxy; ++ix) {
                    double xl = (double)(ix - nr) * p, xh = (double)(ix - nr + 1) * p;
                    double yl = (double)(iy - nr) * p, yh = (double)(iy - nr + 1) * p;
                    int inc = xh > ar[c][0] && xl < ar[c][1] && yh > ar[c][2] && yl < ar[c][3];
                    P->incl[((size_t)(b * 2 + c)) * npsl + (size_t)iy * nxy + ix] = (uint8_t)inc;
                }
        }
    }

    if (!per_psr_n) {
        /* Eq. 3: n = N W / sum over beams, sub-sources, energies, PSLs in A_stype */
        P->n_hist = n_hist;
        double D = 0.0;
        for (int b = 0; b < nb; ++b)
            for (int s = 0; s < 3; ++s)
                for (int e = 0; e < ne; ++e) {
                    const uint8_t *inc = &P->incl[((size_t)(b * 2 + (s ? 1 : 0))) * npsl];
                    const double *W = &P->wpsl[((size_t)s * ne + e) * npsl];
                    D += or_sum32(W, inc, (int64_t)npsl);
                }
        P->denom = D;
        size_t ncnt = (size_t)nb * 3 * ne * npsl;
        double *q = (double *)calloc(ncnt, 8);
        P->count = (int64_t *)calloc(ncnt, 8);
        for (int b = 0; b < nb; ++b)
            for (int s = 0; s < 3; ++s)
                for (int e = 0; e < ne; ++e) {
                    const uint8_t *inc = &P->incl[((size_t)(b * 2 + (s ? 1 : 0))) * npsl];
                    const double *W = &P->wpsl[((size_t)s * ne + e) * npsl];
                    double *qq = &q[(((size_t)b * 3 + s) * ne + e) * npsl];
                    for (size_t j = 0; j < npsl; ++j)
                        qq[j] = (inc[j] && D > 0.0) ? ((double)n_hist * W[j]) / D : 0.0;
                }
        hamilton(q, (int64_t)ncnt, D > 0.0 ? n_hist : 0, P->count);
        free(q);
        int64_t ne_ = 0;
        for (size_t j = 0; j < ncnt; ++j) ne_ += P->count[j] > 0;
        ent_alloc(P, ne_);
        int64_t k = 0, acc = 0;
        for (int b = 0; b < nb; ++b)
            for (int s = 0; s < 3; ++s)
                for (int e = 0; e < ne; ++e)
                    for (int iy = 0; iy < nxy; ++iy)
                        for (int ix = 0; ix < nxy; ++ix) {
                            int64_t c = P->count[(((size_t)b * 3 + s) * ne + e) * npsl + (size_t)iy * nxy + ix];
                            if (c <= 0) continue;
                            P->ent_start[k] = acc; acc += c;
                            P->ent_b[k] = b; P->ent_s[k] = s; P->ent_e[k] = e;
                            P->ent_ix[k] = ix; P->ent_iy[k] = iy; P->ent_tag[k] = -1;
                            ++k;
                        }
        P->ent_start[k] = acc;
        P->n_ent = k;
    } else {
        /* one basis run per (PSR k = (s,e,R), beam b): PSL weights are the k-th
         * share of the conversion; Eq. 3 applied within that run alone */
        P->per_psr = 1;
        int npsr = 3 * ne * nr;
        int64_t cap = 0;
        for (int k = 0; k < npsr; ++k) cap += 1;
        (void)cap;
        /* first pass: count entries */
        size_t maxent = (size_t)npsr * nb * npsl;
        int64_t *cnt_all = (int64_t *)calloc(maxent, 8);
        double *dkb = (double *)calloc((size_t)npsr * nb, 8);
        double *q = (double *)calloc(npsl, 8);
        int64_t *c1 = (int64_t *)calloc(npsl, 8);
        double *wk = (double *)calloc(npsl, 8);
        double *rawk = (double *)calloc(npsl, 8);
        int64_t total = 0;
        for (int k = 0; k < npsr; ++k) {
            int s = k / (ne * nr), e = (k / nr) % ne, R = k % nr;
            const double *W = &M->w[((size_t)s * ne + e) * nr];
            /* the block scale of step 4 for the whole model */
            double sraw = 0.0, sR = 0.0;
            for (int iy = 0; iy < nxy; ++iy)
                for (int ix = 0; ix < nxy; ++ix) {
                    double xc = ((double)(ix - nr) + 0.5) * p, yc = ((double)(iy - nr) + 0.5) * p;
                    double r = sqrt(xc * xc + yc * yc);
                    int r0, in; double l0;
                    ring_interp(r, nr, M->dr, &r0, &l0, &in);
                    double dens = 0.0, dk = 0.0;
                    if (in) {
                        dens = l0 * (W[r0] / M->dr);
                        if (l0 < 1.0) dens += (1.0 - l0) * (W[r0 + 1] / M->dr);
                        if (r0 == R) dk = l0 * (W[R] / M->dr);
                        else if (r0 + 1 == R && l0 < 1.0) dk = (1.0 - l0) * (W[R] / M->dr);
                    }
                    rawk[iy * nxy + ix] = dens / (2.0 * PI_D * r);
                    wk[iy * nxy + ix] = dk / (2.0 * PI_D * r);
                }
            sraw = or_sum32(rawk, NULL, (int64_t)npsl);
            for (int RR = 0; RR < nr; ++RR) sR += W[RR];
            double scale = sraw > 0.0 ? sR / sraw : 0.0;
            for (size_t j = 0; j < npsl; ++j) wk[j] = wk[j] * scale;
            for (int b = 0; b < nb; ++b) {
                const uint8_t *inc = &P->incl[((size_t)(b * 2 + (s ? 1 : 0))) * npsl];
                const double D = or_sum32(wk, inc, (int64_t)npsl);
                dkb[(size_t)k * nb + b] = D;
                for (size_t j = 0; j < npsl; ++j)
                    q[j] = (inc[j] && D > 0.0) ? ((double)per_psr_n[k] * wk[j]) / D : 0.0;
                hamilton(q, (int64_t)npsl, D > 0.0 ? per_psr_n[k] : 0, c1);
                memcpy(&cnt_all[((size_t)k * nb + b) * npsl], c1, npsl * 8);
                for (size_t j = 0; j < npsl; ++j) total += c1[j];
            }
        }
        int64_t ne_ = 0;
        for (size_t j = 0; j < maxent; ++j) ne_ += cnt_all[j] > 0;
        ent_alloc(P, ne_);
        int64_t kk = 0, acc = 0;
        for (int k = 0; k < npsr; ++k)
            for (int b = 0; b < nb; ++b)
                for (int iy = 0; iy < nxy; ++iy)
                    for (int ix = 0; ix < nxy; ++ix) {
                        int64_t c = cnt_all[((size_t)k * nb + b) * npsl + (size_t)iy * nxy + ix];
                        if (c <= 0) continue;
                        P->ent_start[kk] = acc; acc += c;
                        P->ent_b[kk] = b; P->ent_s[kk] = k / (ne * nr); P->ent_e[kk] = (k / nr) % ne;
                        P->ent_ix[kk] = ix; P->ent_iy[kk] = iy; P->ent_tag[kk] = k;
                        P->ent_scale[kk] = dkb[(size_t)k * nb + b] / (double)per_psr_n[k];
                        ++kk;
                    }
        P->ent_start[kk] = acc;
        P->n_ent = kk;
        P->n_hist = acc;
        P->count = cnt_all;   /* [npsr][n_beams][n_xy][n_xy] */
        free(dkb); free(q); free(c1); free(wk); free(rawk);
    }
    return P;
}

/* sizes: [n_xy, n_ent, n_hist, per_psr] and the denominator */
OR_API void or_plan_sizes(const void *h, int64_t out[4], double *denom)
{
    const or_plan *P = (const or_plan *)h;
    out[0] = P->n_xy; out[1] = P->n_ent; out[2] = P->n_hist; out[3] = P->per_psr;
    *denom = P->denom;
}

/* which: 0 wpsl (double [3][n_e][n_xy^2]); 1 incl (u8 [n_beams][2][n_xy^2]);
 * 2 area (double [n_beams][2][4]); 3 count (int64, whole-plan
 * [n_beams][3][n_e][n_xy^2] or per-PSR [n_psr][n_beams][n_xy^2]);
 * 4 ent_start (int64 [n_ent+1]); 5 entries (int32 [n_ent][6]: b s e ix iy tag);
 * 6 ent_scale (double [n_ent]); 7 tag_r0 (int32 [n_xy^2]); 8 tag_l0 (double [n_xy^2]) */
OR_API void or_plan_copy(const void *h, int which, void *dst)
{
    const or_plan *P = (const or_plan *)h;
    size_t npsl = (size_t)P->n_xy * P->n_xy;
    switch (which) {
    case 0: memcpy(dst, P->wpsl, 3 * (size_t)P->n_e * npsl * 8); break;
    case 1: memcpy(dst, P->incl, (size_t)P->n_beams * 2 * npsl); break;
    case 2: memcpy(dst, P->area, (size_t)P->n_beams * 8 * 8); break;
    case 3:
        if (P->per_psr) memcpy(dst, P->count, (size_t)3 * P->n_e * P->n_r * P->n_beams * npsl * 8);
        else memcpy(dst, P->count, (size_t)P->n_beams * 3 * P->n_e * npsl * 8);
        break;
    case 4: memcpy(dst, P->ent_start, (size_t)(P->n_ent + 1) * 8); break;
    case 5: {
        int32_t *o = (int32_t *)dst;
        for (int64_t k = 0; k < P->n_ent; ++k) {
            o[6 * k + 0] = P->ent_b[k]; o[6 * k + 1] = P->ent_s[k]; o[6 * k + 2] = P->ent_e[k];
            o[6 * k + 3] = P->ent_ix[k]; o[6 * k + 4] = P->ent_iy[k]; o[6 * k + 5] = P->ent_tag[k];
        }
        break;
    }
    case 6: memcpy(dst, P->ent_scale, (size_t)(P->n_ent > 0 ? P->n_ent : 0) * 8); break;
    case 7: memcpy(dst, P->tag_r0, npsl * 4); break;
    case 8: memcpy(dst, P->tag_l0, npsl * 8); break;
    default: break;
    }
}

/* ------------------------------------------------------------------------- */
/* Source sampling, steps S3-S5                                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    double x, y, z, u, v, w, E;      /* at the phantom surface plane */
    double xp, yp, up, vp, wp;       /* at the phase-space plane */
    int type;                        /* 0 photon, 1 electron */
    int status;                      /* 0 accepted, 1 rejected by the jaws */
    int stype, ebin, ring, comp, psr, beam;
    int64_t ent;
    double edge;                     /* distance to the nearest jaw edge in the jaw planes */
} or_src;

/* largest entry k with ent_start[k] <= h */
static int64_t find_entry(const or_plan *P, int64_t h)
{
    int64_t lo = 0, hi = P->n_ent - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (P->ent_start[mid] <= h) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* ring holding the sampled position, decided in single precision exactly as a
 * single-precision implementation without fused multiply-add would decide it */
static int ring_of_f32(float xf, float yf, int n_r, double dr)
{
    float r2 = xf * xf + yf * yf;
    float drf = (float)dr;
    int i = 0;
    for (int k = 1; k < n_r; ++k) {
        float ek = (float)k * drf;
        if (r2 >= ek * ek) i = k;
    }
    return i;
}

static uint64_t thresh32(double p)
{
    double t = floor(p * 4294967296.0);
    if (t < 0.0) t = 0.0;
    if (t > 4294967296.0) t = 4294967296.0;
    return (uint64_t)t;
}

static void sample_one(const or_plan *P, uint64_t seed, uint64_t g, double z_surf, or_src *o)
{
    const or_model *M = &P->M;
    int64_t h = (int64_t)(g % (uint64_t)P->n_hist);
    int64_t k = find_entry(P, h);
    int b = P->ent_b[k], s = P->ent_s[k], e = P->ent_e[k], ix = P->ent_ix[k], iy = P->ent_iy[k];
    int nr = P->n_r, nxy = P->n_xy;
    double p = P->p;
    stream_t st;
    stream_init(&st, seed, g, 0u);
    uint32_t a[4], bb[4];
    draw(&st, a);
    draw(&st, bb);

    /* position uniform in the PSL, energy uniform in the bin (S3) */
    double xl = (double)(ix - nr) * p, yl = (double)(iy - nr) * p;
    double x = xl + u01(a[0]) * p;
    double y = yl + u01(a[1]) * p;
    double E = M->e_lo[s] + ((double)e + u01(a[2])) * M->de[s];
    float pf = (float)p;
    float xf = (float)(ix - nr) * pf + u01f(a[0]) * pf;
    float yf = (float)(iy - nr) * pf + u01f(a[1]) * pf;
    int ring = ring_of_f32(xf, yf, nr, M->dr);

    /* Box-Muller pair */
    double rad = sqrt(-2.0 * log(u01(bb[0])));
    double ang = 2.0 * PI_D * u01(bb[1]);
    double n1 = rad * cos(ang), n2 = rad * sin(ang);

    /* PSR index carried for the basis tally */
    int R;
    if (P->ent_tag[k] >= 0) {
        R = P->ent_tag[k] % nr;
    } else {
        int r0 = P->tag_r0[iy * nxy + ix];
        double l0 = P->tag_l0[iy * nxy + ix];
        const double *W = &M->w[((size_t)s * P->n_e + e) * nr];
        R = r0;
        if (l0 < 1.0 && r0 + 1 < nr) {
            double a0 = l0 * W[r0], a1 = (1.0 - l0) * W[r0 + 1];
            double p0 = (a0 + a1) > 0.0 ? a0 / (a0 + a1) : 1.0;
            if (!((uint64_t)bb[2] < thresh32(p0))) R = r0 + 1;
        }
    }

    double u0, v0, w0;
    int comp = -1;
    if (s == 0) {
        /* Eq. 4-5: Gaussian spot, direction from the spot to (r, 0, z_phsp) */
        double xs = M->sigma_s * n1, ys = M->sigma_s * n2;
        double r = sqrt(x * x + y * y);
        double d = sqrt((r - xs) * (r - xs) + ys * ys + M->z_phsp * M->z_phsp);
        u0 = (r - xs) / d; v0 = -ys / d; w0 = M->z_phsp / d;
    } else {
        double al, be;
        size_t pi = ((size_t)e * nr + ring);
        if (s == 1) {
            /* Eq. 6: component from the cumulative table P_{i,k}, then Gaussians */
            const double *c = &M->mix_c[pi * 3];
            double tot = c[0] + c[1] + c[2];
            double P1 = c[0] / tot, P2 = (c[0] + c[1]) / tot;
            if ((uint64_t)a[3] < thresh32(P1)) comp = 0;
            else if ((uint64_t)a[3] < thresh32(P2)) comp = 1;
            else comp = 2;
            al = M->mix_mu[pi * 3 + comp] + M->mix_sa[pi * 3 + comp] * n1;
            be = M->mix_sb[pi * 3 + comp] * n2;
        } else {
            /* Eq. 7 */
            al = M->e_sa[pi] * n1;
            be = M->e_sb[pi] * n2;
        }
        double ta = tan(al), tb = tan(be);   /* alpha = atan(u/w), beta = atan(v/w) */
        double d = sqrt(ta * ta + tb * tb + 1.0);
        u0 = ta / d; v0 = tb / d; w0 = 1.0 / d;
    }
    /* rotate the local (u along the radius) frame by theta = atan2(y, x) */
    double th = atan2(y, x);
    double ct = cos(th), sn = sin(th);
    double u = u0 * ct - v0 * sn, v = u0 * sn + v0 * ct, w = w0;

    /* jaw rejection at the upper jaw surfaces */
    const double *J = &P->jaws[4 * b];
    double zy = P->z_jaw_y, zx = P->z_jaw_x;
    double yJ = y + (zy - M->z_phsp) * v / w;
    double xJ = x + (zx - M->z_phsp) * u / w;
    double ylo = J[2] * zy / P->sad, yhi = J[3] * zy / P->sad;
    double xlo = J[0] * zx / P->sad, xhi = J[1] * zx / P->sad;
    int ok = (yJ >= ylo && yJ <= yhi && xJ >= xlo && xJ <= xhi);
    double edge = fabs(yJ - ylo);
    if (fabs(yJ - yhi) < edge) edge = fabs(yJ - yhi);
    if (fabs(xJ - xlo) < edge) edge = fabs(xJ - xlo);
    if (fabs(xJ - xhi) < edge) edge = fabs(xJ - xhi);

    o->xp = x; o->yp = y; o->up = u; o->vp = v; o->wp = w;
    o->x = x + (z_surf - M->z_phsp) * u / w;
    o->y = y + (z_surf - M->z_phsp) * v / w;
    o->z = z_surf; o->u = u; o->v = v; o->w = w; o->E = E;
    o->type = (s == 2) ? 1 : 0;
    o->status = ok ? 0 : 1;
    o->stype = s; o->ebin = e; o->ring = ring; o->comp = comp;
    o->psr = (s * P->n_e + e) * nr + R;
    o->beam = b; o->ent = k; o->edge = edge;
}

/* Sample histories [g0, g0+n). f64 out [n][12]: x y z u v w E xp yp up vp wp;
 * i32 out [n][9]: type status stype ebin ring comp psr beam entry; edge [n]. */
OR_API int or_sample(const void *h, uint64_t seed, uint64_t g0, int64_t n, double z_surf,
                     double *f64, int32_t *i32, double *edge)
{
    const or_plan *P = (const or_plan *)h;
    if (!P || P->n_ent <= 0) return 1;
    for (int64_t i = 0; i < n; ++i) {
        or_src o;
        sample_one(P, seed, g0 + (uint64_t)i, z_surf, &o);
        double *f = &f64[12 * i];
        f[0] = o.x; f[1] = o.y; f[2] = o.z; f[3] = o.u; f[4] = o.v; f[5] = o.w; f[6] = o.E;
        f[7] = o.xp; f[8] = o.yp; f[9] = o.up; f[10] = o.vp; f[11] = o.wp;
        int32_t *q = &i32[9 * i];
        q[0] = o.type; q[1] = o.status; q[2] = o.stype; q[3] = o.ebin; q[4] = o.ring;
        q[5] = o.comp; q[6] = o.psr; q[7] = o.beam; q[8] = (int32_t)o.ent;
        edge[i] = o.edge;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Transport (stated simplification) and tallies                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, x0, y0, z0;
    const float *rho;
    const uint8_t *mat;
} or_phantom;

typedef struct {
    int32_t electron_mode;   /* 0 local deposition of electron energy, 1 CSDA */
    int32_t tally_mode;      /* 0 energy per voxel, 1 basis [row][psr] */
    int32_t n_batches;
    int32_t compton_only;    /* pin mode: photoelectric and pair switched off */
    double majorant_factor;  /* >= 1 */
    double f_e;              /* max fractional energy loss per CSDA step */
    double s_geo;            /* max CSDA step, cm (<= 0: half the smallest voxel side) */
    int32_t ms_off;          /* pin mode: no multiple-scattering deflection */
    int32_t max_steps;       /* per particle */
    const uint16_t *idx3d;   /* basis mode: 0 none, else row + 1 */
    int32_t n_rows;          /* rows per beam */
    int32_t n_psr;
    int64_t first_batch;     /* pass bt of the run draws the histories of batch first_batch + bt */
} or_opts;

typedef struct {
    double x, y, z, u, v, w, E;
    int type, psr, beam;
    stream_t rng;
    int have;            /* electrons: words 2-3 of the last block are still unused */
    uint32_t hold[2];
} part_t;

typedef struct {
    const or_phantom *Ph;
    const or_opts *O;
    double rho_max[2];
    double *acc;             /* batch accumulator */
    double dep, esc;         /* per-history ledger */
    int64_t n_flight, n_real, n_esteps, n_cap, n_sec;
    part_t *stack; int sp, cap;
    int64_t overflow;
} tctx;

static int voxel_of(const or_phantom *Ph, double x, double y, double z)
{
    double fx = floor((x - Ph->x0) / Ph->dx), fy = floor((y - Ph->y0) / Ph->dy),
           fz = floor((z - Ph->z0) / Ph->dz);
    if (fx < 0 || fy < 0 || fz < 0 || fx >= Ph->nx || fy >= Ph->ny || fz >= Ph->nz) return -1;
    return ((int)fz * Ph->ny + (int)fy) * Ph->nx + (int)fx;
}

static void deposit(tctx *T, int vox, double e, const part_t *p)
{
    if (vox < 0) { T->esc += e; return; }
    T->dep += e;
    if (T->O->tally_mode == 0) {
        T->acc[vox] += e;
    } else {
        int row = T->O->idx3d[vox];
        if (row > 0)
            T->acc[((size_t)p->beam * T->O->n_rows + (row - 1)) * T->O->n_psr + p->psr] += e;
    }
}

static double mu_comp(double E, int m, int comp, const or_opts *O)
{
    if (O->compton_only) return (comp == 0 || comp == 3) ? or_mu_mass(E, m, 0) : 0.0;
    return or_mu_mass(E, m, comp);
}

static double majorant(const tctx *T, double E)
{
    double best = 0.0;
    for (int m = 0; m < 2; ++m) {
        double v = T->rho_max[m] * mu_comp(E, m, 3, T->O);
        if (v > best) best = v;
    }
    return best * T->O->majorant_factor;
}

/* rotate direction (u,v,w) by polar cos(theta) and azimuth phi */
static void rotate_dir(double *u, double *v, double *w, double cost, double phi)
{
    double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
    double cp = cos(phi), sp = sin(phi);
    double un, vn, wn;
    if (fabs(*w) < 0.99999) {
        double s = sqrt(1.0 - (*w) * (*w));
        un = (*u) * cost + sint * ((*u) * (*w) * cp - (*v) * sp) / s;
        vn = (*v) * cost + sint * ((*v) * (*w) * cp + (*u) * sp) / s;
        wn = (*w) * cost - sint * s * cp;
    } else {
        un = sint * cp; vn = sint * sp; wn = ((*w) > 0.0 ? 1.0 : -1.0) * cost;
    }
    double nrm = sqrt(un * un + vn * vn + wn * wn);
    *u = un / nrm; *v = vn / nrm; *w = wn / nrm;
}

static void push(tctx *T, const part_t *p)
{
    if (T->sp >= T->cap) { T->overflow++; return; }
    T->stack[T->sp++] = *p;
}

static void spawn_electron(tctx *T, const part_t *par, double Ee, double u, double v, double w,
                           uint32_t sid, int vox)
{
    if (T->O->electron_mode == 0 || Ee < E_CUT_E) { deposit(T, vox, Ee, par); return; }
    part_t c = *par;
    c.type = 1; c.E = Ee; c.u = u; c.v = v; c.w = w;
    c.rng.sid = sid; c.rng.ctr = 0; c.have = 0;
    if (T->sp < T->cap) T->n_sec++;     /* a secondary electron handed to electron transport */
    push(T, &c);
}

/* Integral from 1 to eta of the Klein-Nishina density of eta = E/E' (up to a
 * constant factor), k = E/mc^2: the density is t^-2 (1/t + t - sin^2 theta)
 * with cos theta = 1 - (t - 1)/k, whose integral has this closed form. */
OR_API double or_kn_cdf(double eta, double k)
{
    double ie = 1.0 / eta, le = log(eta), k1 = k + 1.0;
    return 0.5 * (1.0 - ie * ie) + le + ie - 1.0 + (k1 * k1 * (1.0 - ie) - 2.0 * k1 * le + eta - 1.0) / (k * k);
}

/* Compton sampling by inverting the Klein-Nishina CDF (bisection in FP64):
 * Philox word w_eta -> eta, word w_phi -> azimuth. */
static void kn_sample(uint32_t w_eta, uint32_t w_phi, double k, double *eta_out, double *phi_out)
{
    double emax = 1.0 + 2.0 * k;
    double target = u01(w_eta) * or_kn_cdf(emax, k);
    double lo = 1.0, hi = emax;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        double mid = 0.5 * (lo + hi);
        if (or_kn_cdf(mid, k) < target) lo = mid; else hi = mid;
    }
    *eta_out = 0.5 * (lo + hi);
    *phi_out = 2.0 * PI_D * u01(w_phi);
}

/* One Compton event at photon energy E travelling along (u, v, w): the
 * scattered photon's energy E1 = E / eta and direction d1 (polar cos theta =
 * 1 - (eta - 1) / k about the old direction, azimuth phi), eta drawn from the
 * inverse Klein-Nishina CDF; the recoil electron (kinetic energy E - E1) moves
 * along the momentum the photon gave up, E * u_old - E1 * u_new (photon
 * momenta E / c and E1 / c, so the electron's direction is their difference). */
static void compton_event(uint32_t w_eta, uint32_t w_phi, double E, double u, double v, double w, double *E1,
                          double d1[3], double de[3])
{
    double k = E / ME, eta, phi;
    kn_sample(w_eta, w_phi, k, &eta, &phi);
    double cost = 1.0 - (eta - 1.0) / k;
    double e1 = E / eta;
    double un = u, vn = v, wn = w;
    rotate_dir(&un, &vn, &wn, cost, phi);
    double ex = E * u - e1 * un, ey = E * v - e1 * vn, ez = E * w - e1 * wn;
    double en = sqrt(ex * ex + ey * ey + ez * ez);
    if (en > 0.0) { ex /= en; ey /= en; ez /= en; } else { ex = u; ey = v; ez = w; }
    *E1 = e1;
    d1[0] = un; d1[1] = vn; d1[2] = wn;
    de[0] = ex; de[1] = ey; de[2] = ez;
}

/* Gaussian multiple-scattering deflection after a CSDA step of length ds
 * (cm) through density rho of material m, for an electron of kinetic energy
 * E0 at the start of the step: the step is t = rho ds / X0 radiation lengths,
 * theta0 the Highland width of each projected angle, and the deflection the
 * polar angle of a two-dimensional Gaussian of per-plane width theta0, i.e.
 * theta = theta0 sqrt(-2 ln u1) (Rayleigh), azimuth 2 pi u2.  One Philox block
 * serves two deflections: words 0-1, then words 2-3 at the next one. */
static void ms_deflect(part_t *p, double E0, double rho, double ds, int m)
{
    uint32_t ua, ub;
    if (p->have) {
        ua = p->hold[0]; ub = p->hold[1]; p->have = 0;
    } else {
        uint32_t r[4];
        draw(&p->rng, r);
        ua = r[0]; ub = r[1]; p->hold[0] = r[2]; p->hold[1] = r[3]; p->have = 1;
    }
    double th0 = or_highland(E0, rho * ds / X0G[m]);
    double th = th0 * sqrt(-2.0 * log(u01(ua)));
    if (th > PI_D) th = PI_D;
    rotate_dir(&p->u, &p->v, &p->w, cos(th), 2.0 * PI_D * u01(ub));
}

static void photon_track(tctx *T, part_t *p)
{
    const or_phantom *Ph = T->Ph;
    int steps = 0;
    for (;;) {
        int vox = voxel_of(Ph, p->x, p->y, p->z);
        if (vox < 0) { T->esc += p->E; return; }
        if (p->E < E_CUT_G) { deposit(T, vox, p->E, p); return; }
        if (++steps > T->O->max_steps) { T->n_cap++; deposit(T, vox, p->E, p); return; }
        /* one Philox block per flight: word 0 -> flight length, word 1 ->
         * the collision (virtual, or which interaction), words 2-3 -> a
         * Compton event's eta and azimuth */
        uint32_t r[4];
        draw(&p->rng, r);
        double mumax = majorant(T, p->E);
        double s = -log(u01(r[0])) / mumax;                   /* Woodcock flight */
        p->x += s * p->u; p->y += s * p->v; p->z += s * p->w;
        T->n_flight++;
        vox = voxel_of(Ph, p->x, p->y, p->z);
        if (vox < 0) { T->esc += p->E; return; }
        int m = Ph->mat[vox];
        double rho = (double)Ph->rho[vox];
        double muC = mu_comp(p->E, m, 0, T->O) * rho;
        double muP = mu_comp(p->E, m, 1, T->O) * rho;
        double muQ = mu_comp(p->E, m, 2, T->O) * rho;
        double mut = muC + muP + muQ;
        /* t is uniform on [0, mumax): above mut the collision is virtual;
         * below it t is uniform on [0, mut) and picks the interaction with
         * probabilities muC, muP, muQ over mut */
        double t = u01(r[1]) * mumax;
        if (t > mut) continue;                                /* virtual collision */
        T->n_real++;
        if (t <= muC) {
            double E1, d1[3], de[3];
            compton_event(r[2], r[3], p->E, p->u, p->v, p->w, &E1, d1, de);
            spawn_electron(T, p, p->E - E1, de[0], de[1], de[2], child_id(&p->rng, 0), vox);
            p->E = E1; p->u = d1[0]; p->v = d1[1]; p->w = d1[2];
        } else if (t <= muC + muP) {
            /* photoelectric: the electron takes the photon energy and direction */
            spawn_electron(T, p, p->E, p->u, p->v, p->w, child_id(&p->rng, 0), vox);
            return;
        } else {
            /* pair: uniform kinetic split, both leptons along the photon; the
             * positron is transported as an electron and its annihilation
             * photons leave the interaction point back to back, isotropic */
            uint32_t q[4];
            draw(&p->rng, q);
            double Tk = p->E - 2.0 * ME;
            double Tm = u01(q[0]) * Tk, Tp = Tk - Tm;
            double ca = 2.0 * u01(q[1]) - 1.0, pa = 2.0 * PI_D * u01(q[2]);
            double sa = sqrt(fmax(0.0, 1.0 - ca * ca));
            double ax = sa * cos(pa), ay = sa * sin(pa), az = ca;
            uint32_t ids[4];
            for (uint32_t c = 0; c < 4; ++c) ids[c] = child_id(&p->rng, c);
            spawn_electron(T, p, Tm, p->u, p->v, p->w, ids[0], vox);
            spawn_electron(T, p, Tp, p->u, p->v, p->w, ids[1], vox);
            part_t g = *p;
            g.type = 0; g.E = ME; g.rng.ctr = 0; g.have = 0;
            g.u = ax; g.v = ay; g.w = az; g.rng.sid = ids[2];
            push(T, &g);
            g.u = -ax; g.v = -ay; g.w = -az; g.rng.sid = ids[3];
            push(T, &g);
            return;
        }
    }
}

static void electron_track(tctx *T, part_t *p)
{
    const or_phantom *Ph = T->Ph;
    const or_opts *O = T->O;
    double sgeo = O->s_geo > 0.0 ? O->s_geo
                                  : 0.5 * fmin(Ph->dx, fmin(Ph->dy, Ph->dz));
    int steps = 0;
    for (;;) {
        int vox = voxel_of(Ph, p->x, p->y, p->z);
        if (vox < 0) { T->esc += p->E; return; }
        if (p->E < E_CUT_E || O->electron_mode == 0) { deposit(T, vox, p->E, p); return; }
        if (++steps > O->max_steps) { T->n_cap++; deposit(T, vox, p->E, p); return; }
        int m = Ph->mat[vox];
        double rho = (double)Ph->rho[vox];
        double S = or_scol_mass(p->E, m) * rho;                /* MeV/cm */
        double ds = O->f_e * p->E / S;
        if (ds > sgeo) ds = sgeo;
        double Emid = p->E - 0.5 * S * ds;                     /* midpoint rule */
        double dE = or_scol_mass(Emid, m) * rho * ds;
        if (dE > p->E) dE = p->E;
        int vm = voxel_of(Ph, p->x + 0.5 * ds * p->u, p->y + 0.5 * ds * p->v,
                          p->z + 0.5 * ds * p->w);
        deposit(T, vm, dE, p);
        T->n_esteps++;
        double E0 = p->E;
        p->x += ds * p->u; p->y += ds * p->v; p->z += ds * p->w;
        p->E -= dE;
        if (p->E >= E_CUT_E && !O->ms_off) ms_deflect(p, E0, rho, ds, m);
    }
}

/*
 * Run n_batches passes over the plan (histories g = (first_batch + b) * n_hist + h:
 * a run of B batches equals runs over disjoint batch ranges, summed).
 * s1/s2: per tally cell, the sum over batches of the batch total and of its
 * square (energy in MeV). ledger[4]: source, rejected, escaped (incl. missing
 * the phantom), deposited energy. stats[9]: histories, accepted photons,
 * accepted electrons, rejected, missed, Woodcock flights, real interactions,
 * electron steps, secondary electrons (those photon interactions hand to
 * electron transport). cons[2]: max per-history |balance| / E_source, step-cap hits.
 * per_hist (may be NULL): [n_batches*n_hist] energy deposited per history.
 */
/*
 * Gantry rotation of a beam (the plan's beam geometry): a beam-frame point q
 * (target at the origin, axis +z, isocentre at (0, 0, sad)) lies at
 * iso + R (q - (0, 0, sad)) in phantom coordinates, R turning by the gantry
 * angle g about y: R (a, b, c) = (a cos g + c sin g, b, -a sin g + c cos g).
 * The particle leaves the phase-space plane at (xp, yp, z_phsp) along
 * (u, v, w) and enters the phantom where that straight line first meets the
 * voxel box (Kay-Kajiya slabs); it starts 1e-4 cm past that point.
 * Returns 0 and fills pos/dir (phantom coordinates), or 1 on a miss.
 */
OR_API int or_beam_entry(const double iso[3], double sad, double z_phsp, double g, const double p_plane[2],
                         const double dir[3], const double box_lo[3], const double box_hi[3], double pos[3],
                         double d[3])
{
    double c = cos(g), sn = sin(g);
    double qx = p_plane[0], qy = p_plane[1], qz = z_phsp - sad;
    double p[3] = {iso[0] + qx * c + qz * sn, iso[1] + qy, iso[2] - qx * sn + qz * c};
    d[0] = dir[0] * c + dir[2] * sn; d[1] = dir[1]; d[2] = -dir[0] * sn + dir[2] * c;
    double tn = 0.0, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0) {
            double t1 = (box_lo[a] - p[a]) / d[a], t2 = (box_hi[a] - p[a]) / d[a];
            double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
            if (lo > tn) tn = lo;
            if (hi < tf) tf = hi;
        } else if (p[a] < box_lo[a] || p[a] > box_hi[a]) {
            return 1;
        }
    }
    if (!(tn <= tf)) return 1;
    double t = tn + 1e-4;
    for (int a = 0; a < 3; ++a) pos[a] = p[a] + t * d[a];
    return 0;
}

OR_API int or_run(const void *h, const or_phantom *Ph, const or_opts *O, uint64_t seed,
                  double *s1, double *s2, double *ledger, int64_t *stats, double *cons,
                  double *per_hist)
{
    const or_plan *P = (const or_plan *)h;
    if (!P || P->n_ent <= 0 || O->n_batches < 1 || O->first_batch < 0) return 1;
    size_t nvox = (size_t)Ph->nx * Ph->ny * Ph->nz;
    size_t ncell = O->tally_mode == 0 ? nvox : (size_t)P->n_beams * O->n_rows * O->n_psr;
    tctx T;
    memset(&T, 0, sizeof(T));
    T.Ph = Ph; T.O = O;
    for (size_t v = 0; v < nvox; ++v) {
        int m = Ph->mat[v];
        if ((double)Ph->rho[v] > T.rho_max[m]) T.rho_max[m] = (double)Ph->rho[v];
    }
    T.acc = (double *)calloc(ncell, 8);
    T.cap = 1 << 16;
    T.stack = (part_t *)malloc(sizeof(part_t) * (size_t)T.cap);
    memset(s1, 0, ncell * 8); memset(s2, 0, ncell * 8);
    memset(ledger, 0, 4 * 8); memset(stats, 0, 8 * 8);
    cons[0] = 0.0; cons[1] = 0.0;
    double *batch_scale = NULL;
    (void)batch_scale;
    for (int bt = 0; bt < O->n_batches; ++bt) {
        for (int64_t hh = 0; hh < P->n_hist; ++hh) {
            uint64_t g = (uint64_t)(O->first_batch + bt) * (uint64_t)P->n_hist + (uint64_t)hh;
            or_src o;
            sample_one(P, seed, g, Ph->z0, &o);
            stats[0]++;
            ledger[0] += o.E;
            T.dep = 0.0; T.esc = 0.0;
            double rej = 0.0;
            if (o.status) { rej = o.E; stats[3]++; }
            else {
                part_t p;
                p.x = o.x; p.y = o.y; p.z = o.z; p.u = o.u; p.v = o.v; p.w = o.w; p.E = o.E;
                p.type = o.type; p.psr = o.psr; p.beam = o.beam;
                stream_init(&p.rng, seed, g, 1u);
                p.have = 0;
                int vox = -1;
                if (!P->rotated) {
                    vox = voxel_of(Ph, p.x, p.y, p.z);
                } else {
                    double lo[3] = {Ph->x0, Ph->y0, Ph->z0};
                    double hi[3] = {Ph->x0 + Ph->nx * Ph->dx, Ph->y0 + Ph->ny * Ph->dy, Ph->z0 + Ph->nz * Ph->dz};
                    double pp[2] = {o.xp, o.yp}, dir[3] = {o.up, o.vp, o.wp}, pos[3], d[3];
                    if (or_beam_entry(P->iso, P->sad, P->M.z_phsp, P->gantry[o.beam], pp, dir, lo, hi, pos, d) == 0) {
                        p.x = pos[0]; p.y = pos[1]; p.z = pos[2]; p.u = d[0]; p.v = d[1]; p.w = d[2];
                        vox = voxel_of(Ph, p.x, p.y, p.z);
                    }
                }
                if (vox < 0) { T.esc += p.E; stats[4]++; }
                else {
                    if (p.type) stats[2]++; else stats[1]++;
                    double scale = P->per_psr ? P->ent_scale[o.ent] : 0.0;
                    (void)scale;
                    T.sp = 0;
                    push(&T, &p);
                    while (T.sp > 0) {
                        part_t q = T.stack[--T.sp];
                        if (q.type == 0) photon_track(&T, &q); else electron_track(&T, &q);
                    }
                }
            }
            ledger[1] += rej; ledger[2] += T.esc; ledger[3] += T.dep;
            double bal = fabs(o.E - (rej + T.esc + T.dep)) / o.E;
            if (bal > cons[0]) cons[0] = bal;
            if (per_hist) per_hist[(int64_t)bt * P->n_hist + hh] = T.dep;
        }
        for (size_t c = 0; c < ncell; ++c) {
            s1[c] += T.acc[c];
            s2[c] += T.acc[c] * T.acc[c];
            T.acc[c] = 0.0;
        }
    }
    stats[5] = T.n_flight; stats[6] = T.n_real; stats[7] = T.n_esteps; stats[8] = T.n_sec;
    cons[1] = (double)T.n_cap + (double)T.overflow * 1e6;
    free(T.acc); free(T.stack);
    return 0;
}

/* Pin helper: monoenergetic pencil photons along +z entering a phantom at its
 * top-face centre; returns the depth below the surface of the first real
 * interaction (or -1 when the photon leaves), using the same flight code. */
OR_API void or_first_collision(const or_phantom *Ph, const or_opts *O, double E, uint64_t seed,
                               int64_t n, double *depth)
{
    tctx T;
    memset(&T, 0, sizeof(T));
    T.Ph = Ph; T.O = O;
    size_t nvox = (size_t)Ph->nx * Ph->ny * Ph->nz;
    for (size_t v = 0; v < nvox; ++v) {
        int m = Ph->mat[v];
        if ((double)Ph->rho[v] > T.rho_max[m]) T.rho_max[m] = (double)Ph->rho[v];
    }
    double xc = Ph->x0 + 0.5 * Ph->nx * Ph->dx, yc = Ph->y0 + 0.5 * Ph->ny * Ph->dy;
    for (int64_t i = 0; i < n; ++i) {
        part_t p;
        p.x = xc; p.y = yc; p.z = Ph->z0; p.u = 0; p.v = 0; p.w = 1; p.E = E;
        stream_init(&p.rng, seed, (uint64_t)i, 1u);
        p.have = 0;
        depth[i] = -1.0;
        for (;;) {
            uint32_t r[4];
            draw(&p.rng, r);
            double mumax = majorant(&T, p.E);
            p.z += -log(u01(r[0])) / mumax;
            int vox = voxel_of(Ph, p.x, p.y, p.z);
            if (vox < 0) break;
            double mut = mu_comp(p.E, Ph->mat[vox], 3, O) * (double)Ph->rho[vox];
            if (u01(r[1]) * mumax > mut) continue;
            depth[i] = p.z - Ph->z0;
            break;
        }
    }
}

/* Pin helper: n Compton events at energy E through the same inverse-CDF sampler
 * (words 2-3 of a fresh block, as in a flight); out [n][2] = (E'/E, cos theta). */
OR_API void or_kn_samples(double E, uint64_t seed, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        stream_t st;
        stream_init(&st, seed, (uint64_t)i, 1u);
        uint32_t r[4];
        draw(&st, r);
        double k = E / ME, eta, phi;
        kn_sample(r[2], r[3], k, &eta, &phi);
        out[2 * i] = 1.0 / eta;
        out[2 * i + 1] = 1.0 - (eta - 1.0) / k;
    }
}

/* Pin helper: one electron of energy E along +z from the top-face centre with
 * the run's CSDA stepping; returns path length travelled until the cutoff (or
 * escape) and the energy deposited. */
OR_API void or_electron_path(const or_phantom *Ph, const or_opts *O, double E, uint64_t seed,
                             double out[2])
{
    tctx T;
    memset(&T, 0, sizeof(T));
    T.Ph = Ph; T.O = O;
    part_t p;
    p.x = Ph->x0 + 0.5 * Ph->nx * Ph->dx; p.y = Ph->y0 + 0.5 * Ph->ny * Ph->dy;
    p.z = Ph->z0 + 1e-9; p.u = 0; p.v = 0; p.w = 1; p.E = E; p.type = 1; p.psr = 0; p.beam = 0;
    stream_init(&p.rng, seed, 0, 1u);
    p.have = 0;
    double z0 = p.z;
    /* tally_mode 0 with a scratch accumulator */
    size_t nvox = (size_t)Ph->nx * Ph->ny * Ph->nz;
    T.acc = (double *)calloc(nvox, 8);
    electron_track(&T, &p);
    out[0] = p.z - z0;
    out[1] = T.dep;
    free(T.acc);
}

/* Pin helper: n Compton events of photons of energy E along d0 through the
 * transport's own event code (history i, primary transport stream; eta and
 * azimuth from words 2-3 of the stream's first block, as in a flight); out
 * [n][8] = (E1, photon direction[3], electron kinetic energy, electron
 * direction[3]). */
OR_API void or_compton_events(double E, const double d0[3], uint64_t seed, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        stream_t st;
        stream_init(&st, seed, (uint64_t)i, 1u);
        uint32_t r[4];
        draw(&st, r);
        double E1, d1[3], de[3];
        compton_event(r[2], r[3], E, d0[0], d0[1], d0[2], &E1, d1, de);
        double *o = out + 8 * i;
        o[0] = E1; o[1] = d1[0]; o[2] = d1[1]; o[3] = d1[2];
        o[4] = E - E1; o[5] = de[0]; o[6] = de[1]; o[7] = de[2];
    }
}

/* Pin helper: n independent multiple-scattering deflections (history i) of an
 * electron of energy E0 moving along d0 after one step of length ds through
 * density rho of material m, through the transport's own deflection code;
 * out [n][3] = new direction.  Each uses the first half of a fresh block. */
OR_API void or_ms_deflections(double E0, double rho, double ds, int m, const double d0[3],
                              uint64_t seed, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        part_t p;
        memset(&p, 0, sizeof(p));
        p.u = d0[0]; p.v = d0[1]; p.w = d0[2]; p.E = E0; p.type = 1;
        stream_init(&p.rng, seed, (uint64_t)i, 1u);
        p.have = 0;
        ms_deflect(&p, E0, rho, ds, m);
        out[3 * i] = p.u; out[3 * i + 1] = p.v; out[3 * i + 2] = p.w;
    }
}
