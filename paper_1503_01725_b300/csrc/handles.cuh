// handles.cuh -- layouts of the opaque handles of liblsm.so.
#pragma once

#include "common.cuh"

namespace lsm {

// One plan entry: a PSL with a non-zero particle count (16 bytes).
struct EntryRec {
    uint16_t ix, iy;
    uint8_t beam, stype;
    uint16_t ebin;
    int16_t fixed_ring;   // ring carried as PSR index; -1: drawn from (r0, r0 + 1)
    uint8_t r0, pad;
    uint32_t thr;         // drawn tag: ring r0 when the draw < thr, else r0 + 1
};

// Everything the sampling kernels read, passed by value.
struct SampleParams {
    const int64_t *start;      // [n_ent + 1]
    const EntryRec *ent;       // [n_ent]
    const unsigned long long *mixthr;  // [n_e][n_r][2]
    const float4 *mix;         // [n_e][n_r][3] (mu, sigma_alpha, sigma_beta, 0)
    const float2 *esig;        // [n_e][n_r]
    const float *jaws_f;       // [n_beams][4] jaw limits in the jaw planes: ylo yhi xlo xhi
    const int64_t *n_ent;      // device: entries of the plan (written by the build's last scan)
    int n_e, n_r;
    float pitch, z_phsp, sigma_s;
    float e_lo[3], de[3];
    float zy_rel, zx_rel;      // jaw plane minus phase-space plane
    // gantry rotation (rotated != 0): per beam (cos g, sin g), the isocentre
    // in phantom coordinates and the source-to-isocentre distance
    const float2 *rot;
    float iso[3], sad;
    int rotated;
};

// What a captured run graph depends on besides the seed.
struct GraphKey {
    uint64_t psl, ph;     // creation ids of the plan and the phantom
    const void *part, *ws, *batch, *ws2;
    lsm_run_opts o;
    int timed;            // captured with the event timers on
};

// One record of a PSL particle file: a particle on the phase-space plane.
struct PslRec {
    float x, y, u, v, w, E;
    uint32_t tag;         // PSR index | particle type << 16 (0 photon, 1 electron)
    uint32_t info;        // sub-source | energy bin << 8
};
static_assert(sizeof(PslRec) == 32, "PSL file record layout");

// Jaw test and flight to the phantom of PSL-file particles for one beam.
struct PslGeom {
    float jaw[4];         // ylo, yhi, xlo, xhi of the opening on the upper jaw surfaces
    float zy_rel, zx_rel; // upper jaw surfaces - phase-space plane
    float z_rel;          // phantom surface - phase-space plane
    float x0, y0;         // phantom corner on the surface plane
};

}  // namespace lsm

// A validated PSR model (lsm_model_create): a library-owned host copy of the
// caller's arrays, which the plan builds read.
struct lsm_model {
    lsm_psr_model m;      // array pointers point into `data`
    double *data;
};

struct lsm_psl {
    int device;
    uint64_t uid;         // unique per created plan (graph-cache key; addresses can be reused)
    void *arena;          // every device array below lives in this one allocation
    int n_e, n_r, n_xy, n_beams, per_psr;
    double dr, z_phsp, sigma_s, e_lo[3], de[3];
    double sad, z_jaw_y, z_jaw_x;
    int rotated;
    double gantry[16], iso[3];
    // the build's results (denominator, floor sum, n_ent, total) land in
    // h_res (pinned) when event `done` completes; `resolved` once read
    void *done;
    int64_t *h_res;
    int resolved, empty;
    double denom;
    int64_t plan_size, n_ent, ncell;
    double *d_w, *d_wpsl, *d_scale, *d_jaws, *d_area, *d_escale;
    uint8_t *d_incl;
    int64_t *d_count, *d_start;
    lsm::EntryRec *d_ent;
    unsigned long long *d_mixthr;
    float4 *d_mix;
    float2 *d_esig;
    float *d_jaws_f;
    int32_t *d_tag_r0;
    double *d_tag_l0;
    lsm::SampleParams sp;
};

struct lsm_phantom {
    int device;
    uint64_t uid;         // unique per created phantom
    int nx, ny, nz;
    double dx, dy, dz, x0, y0, z0;
    float *d_rho;         // density
    uint8_t *d_mat;
    float *d_rhomat;      // density, negated for material class 1 (one load per voxel)
    double *d_inv_mass;   // 1 / (rho V) per voxel (g^-1): the dose is the deposit times it
    float4 *d_xs;         // [2][kGrid]
    float *d_mumax;       // [kGrid] majorant at factor 1
    unsigned *d_flags;    // [0..1] largest density per material (float bits), [2] nonzero: invalid input
    int validated;        // 1: the input was checked on the host at creation (0: lsm_phantom_create_async)
    double rho_max[2];
};

struct lsm_tally {
    int device;
    int mode, n_rows, n_psr, n_beams;
    int64_t ncell, nvox;
    float *d_part;        // FP32 partials of the current iteration, part_slots slices of ncell
    int part_slots;
    double *d_batch;      // FP64 open batch
    double *d_s1, *d_s2;
    uint16_t *d_idx;      // basis mode
    lsm::RunStats *d_stats;
    int n_batches;
    void *ws;             // cached particle queues of lsm_run / lsm_transport
    uint32_t ws_chunk, ws_ecap;
    void *ws2;            // queues of the second half-iteration (lsm_run_opts.streams = 2)
    uint32_t ws2_chunk, ws2_ecap;
    void *pstream;        // its stream, and the fork and join events
    void *pev[2];
    void *gexec;          // captured run graph (cudaGraphExec_t) and what it was captured for
    lsm::GraphKey gkey;
    int64_t graph_kernels;
    void *gstream;        // stream of graph capture and replay, and its two events
    void *gev[2];
    void *gtimers;        // event timers inside the graph (when captured with timing on)
    double *hl;           // per-history energy ledger (test mode; caller's device buffer) or null
    uint64_t hl_g0;       // history of its entry 0
    int64_t hl_n;         // histories it holds
};
