// PSL files: the comparator source model of Table 1 (Sec. 3.1). Particles are
// stored on disk grouped by phase-spacelet (PSL cell); a dose calculation for
// a field reads the records of the cells its sampling areas include, copies
// them to the GPU and translates them there (jaw test, flight to the
// phantom), then transports them like sampled particles.
//
// Pipeline of lsm_pslfile_run: a reader thread fills three pinned host
// buffers with pread (each chunk split over four threads); the calling thread copies each filled buffer to one of
// two device buffers on a copy stream and queues the enqueue + transport
// kernels of that chunk on the caller's stream, so that the disk read of
// chunk c+1, the copy of chunk c and the transport of chunk c-1 overlap.
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <errno.h>
#include <math.h>
#include <mutex>
#include <string.h>
#include <thread>
#include <vector>

#include "handles.cuh"

namespace lsm {
lsm_status sample_public(const lsm_psl *, uint64_t, uint64_t, int64_t, double, const lsm_particles *, cudaStream_t);
lsm_status resolve_psl(lsm_psl *);
struct PslFileRun;
lsm_status pslfile_begin(const lsm_phantom *, lsm_tally *, const lsm_run_opts *, int64_t, int, uint64_t,
                         cudaStream_t, PslFileRun **);
lsm_status pslfile_chunk(PslFileRun *, const void *, int64_t, uint64_t, int64_t, const PslGeom &, cudaStream_t);
lsm_status pslfile_end_pass(PslFileRun *, cudaStream_t);
lsm_status pslfile_finish(PslFileRun *, cudaStream_t);
}  // namespace lsm

using namespace lsm;

namespace {

constexpr size_t kAlign = 4096;

struct FileHeader {
    char magic[8];
    uint32_t version, record_bytes;
    int32_t n_xy, n_e, n_r, zero;
    double dr, z_phsp, w_record, denom;
    int64_t n_records, index_offset, data_offset;
    uint64_t seed;
};
static_assert(sizeof(FileHeader) == 96, "PSL file header layout");
const char kMagic[8] = {'L', 'S', 'M', 'P', 'S', 'L', 'F', '1'};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// full-length pwrite/pread (the kernel may transfer less than asked)
bool write_all(int fd, const void *p, size_t n, off_t off)
{
    const char *c = (const char *)p;
    while (n) {
        const ssize_t k = pwrite(fd, c, std::min<size_t>(n, (size_t)1 << 30), off);
        if (k < 0 && errno == EINTR) continue;
        if (k <= 0) return false;
        c += k; n -= (size_t)k; off += k;
    }
    return true;
}

bool read_all(int fd, void *p, size_t n, off_t off)
{
    char *c = (char *)p;
    while (n) {
        const ssize_t k = pread(fd, c, std::min<size_t>(n, (size_t)1 << 30), off);
        if (k < 0 && errno == EINTR) continue;
        if (k <= 0) return false;
        c += k; n -= (size_t)k; off += k;
    }
    return true;
}

struct Fd {
    int fd = -1;
    ~Fd() { if (fd >= 0) close(fd); }
};

// Pinned host and device chunk buffers, kept between runs (allocating and
// pinning hundreds of MB costs more than reading a small field's records).
struct BufferPool {
    std::mutex m;
    void *h[3] = {nullptr, nullptr, nullptr};
    void *d[2] = {nullptr, nullptr};
    size_t bytes = 0;
    lsm_status get(size_t need)
    {
        if (bytes >= need) return LSM_OK;
        for (auto &p : h) { if (p) cudaFreeHost(p); p = nullptr; }
        for (auto &p : d) { if (p) cudaFree(p); p = nullptr; }
        bytes = 0;
        for (auto &p : h) LSM_CUDA(cudaMallocHost(&p, need));
        for (auto &p : d) LSM_CUDA(cudaMalloc(&p, need));
        bytes = need;
        return LSM_OK;
    }
};
BufferPool g_pool;

// Records [a, b) of a chunk buffer: piece `buf` of a segment comes from file
// record `file` on. Returns 0 or the failing read's errno.
struct Seg {
    int64_t buf, file, n;
};
constexpr int kReadThreads = 4;

int read_share(int fd, int64_t data_off, const std::vector<Seg> &segs, char *dst, int64_t a, int64_t b)
{
    for (const Seg &s : segs) {
        const int64_t lo = std::max(a, s.buf), hi = std::min(b, s.buf + s.n);
        if (lo >= hi) continue;
        if (!read_all(fd, dst + lo * 32, (size_t)(hi - lo) * 32, (off_t)(data_off + (s.file + lo - s.buf) * 32)))
            return errno ? errno : EIO;
    }
    return 0;
}

// A chunk as the reader thread hands it over.
struct Chunk {
    int64_t n = 0, i0 = 0;
    uint64_t g0 = 0;
    bool end_of_pass = false;
};

}  // namespace

extern "C" lsm_status lsm_pslfile_write(const lsm_psl *P, uint64_t seed, const char *path, int64_t *n_written,
                                        lsm_stream stream)
{
    if (!P || !path) return set_arg_error("lsm_pslfile_write: NULL argument");
    if (P->per_psr || P->n_beams != 1) return set_arg_error("lsm_pslfile_write: needs a whole-source single-beam plan");
    {
        const lsm_status r = resolve_psl(const_cast<lsm_psl *>(P));
        if (r) return r;
    }
    const int64_t M = P->plan_size;
    if (M < 1 || M > ((int64_t)1 << 28)) return set_arg_error("lsm_pslfile_write: 1 <= plan size <= 2^28");
    cudaStream_t st = (cudaStream_t)stream;
    const int nxy = P->n_xy;
    const int64_t npsl = (int64_t)nxy * nxy, ncell = 3 * npsl;
    LSM_CUDA(cudaDeviceSynchronize());
    std::vector<EntryRec> ent((size_t)P->n_ent);
    std::vector<int64_t> start((size_t)P->n_ent + 1);
    LSM_CUDA(cudaMemcpy(ent.data(), P->d_ent, ent.size() * sizeof(EntryRec), cudaMemcpyDeviceToHost));
    LSM_CUDA(cudaMemcpy(start.data(), P->d_start, start.size() * 8, cudaMemcpyDeviceToHost));
    // cell ranges of the file, and where each plan entry's records go in it
    std::vector<int64_t> cstart((size_t)ncell + 1, 0), fill((size_t)ncell, 0), fo((size_t)P->n_ent);
    auto cell_of = [&](const EntryRec &e) { return ((int64_t)e.stype * nxy + e.iy) * nxy + e.ix; };
    for (int64_t k = 0; k < P->n_ent; ++k) cstart[(size_t)cell_of(ent[k]) + 1] += start[k + 1] - start[k];
    for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    for (int64_t k = 0; k < P->n_ent; ++k) {   // plan order: within a cell, energy bins ascend
        const int64_t c = cell_of(ent[k]);
        fo[k] = cstart[c] + fill[c];
        fill[c] += start[k + 1] - start[k];
    }
    if (cstart[ncell] != M) return set_arg_error("lsm_pslfile_write: plan counts do not add up to the plan size");

    std::vector<PslRec> out((size_t)M);
    const int64_t CH = std::min<int64_t>(M, (int64_t)1 << 22);
    // device SoA for the sampler and pinned host copies of the fields kept
    const size_t f4 = (size_t)CH * 4;
    char *dbase = nullptr, *hbase = nullptr;
    const size_t dbytes = 7 * f4 + (size_t)CH * 8 + (size_t)CH * 2 + 3 * (size_t)CH + (size_t)CH * 16 + 4096;   // + 256-byte padding of 12 arrays
    LSM_CUDA(cudaMalloc(&dbase, dbytes));
    cudaError_t ce = cudaMallocHost(&hbase, 6 * f4 + (size_t)CH * 16 + (size_t)CH * 2 + (size_t)CH);
    if (ce != cudaSuccess) { cudaFree(dbase); return set_cuda_error(ce, "lsm_pslfile_write: pinned buffer"); }
    lsm_particles d;
    char *p = dbase;
    float **fl[7] = {&d.x, &d.y, &d.z, &d.u, &d.v, &d.w, &d.E};
    for (auto f : fl) { *f = (float *)p; p += round_up(f4, 256); }
    d.hist = (uint64_t *)p; p += round_up((size_t)CH * 8, 256);
    d.psr = (uint16_t *)p; p += round_up((size_t)CH * 2, 256);
    d.beam = (uint8_t *)p; p += round_up((size_t)CH, 256);
    d.type = (uint8_t *)p; p += round_up((size_t)CH, 256);
    d.status = (uint8_t *)p; p += round_up((size_t)CH, 256);
    d.info = (int32_t *)p;
    float *hf[6];
    for (int k = 0; k < 6; ++k) hf[k] = (float *)(hbase + k * f4);
    int32_t *hinfo = (int32_t *)(hbase + 6 * f4);
    uint16_t *hpsr = (uint16_t *)(hinfo + 4 * CH);
    uint8_t *htype = (uint8_t *)(hpsr + CH);
    lsm_status rc = LSM_OK;
    const float *df[6] = {d.x, d.y, d.u, d.v, d.w, d.E};
    for (int64_t h0 = 0; h0 < M && rc == LSM_OK; h0 += CH) {
        const int64_t n = std::min(CH, M - h0);
        rc = sample_public(P, seed, (uint64_t)h0, n, P->z_phsp, &d, st);
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 6 && rc == LSM_OK && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(hf[k], df[k], (size_t)n * 4, cudaMemcpyDeviceToHost, st);
        if (rc == LSM_OK && e == cudaSuccess) e = cudaMemcpyAsync(hpsr, d.psr, (size_t)n * 2, cudaMemcpyDeviceToHost, st);
        if (rc == LSM_OK && e == cudaSuccess) e = cudaMemcpyAsync(htype, d.type, (size_t)n, cudaMemcpyDeviceToHost, st);
        if (rc == LSM_OK && e == cudaSuccess) e = cudaMemcpyAsync(hinfo, d.info, (size_t)n * 16, cudaMemcpyDeviceToHost, st);
        if (rc == LSM_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (rc == LSM_OK && e != cudaSuccess) rc = set_cuda_error(e, "lsm_pslfile_write: sampling");
        if (rc) break;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t k = hinfo[4 * i + 3];
            const int64_t h = h0 + i;
            if (k < 0 || k >= P->n_ent || h < start[k] || h >= start[k + 1]) {
                rc = set_arg_error("lsm_pslfile_write: sampler entry outside the plan");
                break;
            }
            PslRec &r = out[(size_t)(fo[k] + (h - start[k]))];
            r.x = hf[0][i]; r.y = hf[1][i]; r.u = hf[2][i]; r.v = hf[3][i]; r.w = hf[4][i]; r.E = hf[5][i];
            r.tag = (uint32_t)hpsr[i] | ((uint32_t)htype[i] << 16);
            r.info = (uint32_t)hinfo[4 * i + 0];
        }
    }
    cudaFreeHost(hbase);
    cudaFree(dbase);
    if (rc) return rc;

    FileHeader H;
    memset(&H, 0, sizeof(H));
    memcpy(H.magic, kMagic, 8);
    H.version = 1; H.record_bytes = 32;
    H.n_xy = nxy; H.n_e = P->n_e; H.n_r = P->n_r;
    H.dr = P->dr; H.z_phsp = P->z_phsp; H.denom = P->denom; H.w_record = P->denom / (double)M;
    H.n_records = M; H.index_offset = (int64_t)kAlign;
    H.data_offset = (int64_t)round_up(kAlign + (size_t)(ncell + 1) * 8, kAlign);
    H.seed = seed;
    std::vector<char> head((size_t)H.data_offset, 0);
    memcpy(head.data(), &H, sizeof(H));
    memcpy(head.data() + kAlign, cstart.data(), (size_t)(ncell + 1) * 8);
    Fd f;
    f.fd = open(path, O_WRONLY | O_CREAT | O_TRUNC, 0644);
    if (f.fd < 0) return set_io_error("lsm_pslfile_write: open", path, errno);
    if (!write_all(f.fd, head.data(), head.size(), 0) ||
        !write_all(f.fd, out.data(), out.size() * sizeof(PslRec), (off_t)H.data_offset) || fdatasync(f.fd) != 0)
        return set_io_error("lsm_pslfile_write: write", path, errno);
    if (n_written) *n_written = M;
    return LSM_OK;
}

extern "C" lsm_status lsm_pslfile_run(const char *path, const lsm_psl *field, const lsm_phantom *ph, lsm_tally *t,
                                      uint64_t seed, int32_t n_batches, int32_t n_passes, int32_t cold,
                                      const lsm_run_opts *opts, lsm_pslfile_stats *stats, lsm_stream stream)
{
    const double t_start = now_s();
    if (!path || !field || !ph || !t || !opts) return set_arg_error("lsm_pslfile_run: NULL argument");
    if (n_batches < 1 || n_batches > 255) return set_arg_error("lsm_pslfile_run: 1 <= n_batches <= 255");
    if (n_passes < 1) return set_arg_error("lsm_pslfile_run: n_passes >= 1");
    if (field->per_psr || field->n_beams != 1 || field->rotated)
        return set_arg_error("lsm_pslfile_run: the field must be a whole-source single-beam plan without gantry");
    cudaStream_t st = (cudaStream_t)stream;
    Fd f;
    f.fd = open(path, O_RDONLY);
    if (f.fd < 0) return set_io_error("lsm_pslfile_run: open", path, errno);
    FileHeader H;
    if (!read_all(f.fd, &H, sizeof(H), 0)) return set_io_error("lsm_pslfile_run: header", path, errno);
    if (memcmp(H.magic, kMagic, 8) != 0 || H.version != 1 || H.record_bytes != 32)
        return set_arg_error("lsm_pslfile_run: not a PSL file (magic/version/record size)");
    const int nxy = H.n_xy;
    if (nxy != field->n_xy || !(fabs(H.dr - field->dr) <= 1e-12 * field->dr) ||
        !(fabs(H.z_phsp - field->z_phsp) <= 1e-9 * field->z_phsp))
        return set_arg_error("lsm_pslfile_run: the file's PSL grid or phase-space plane differs from the field's");
    const int64_t npsl = (int64_t)nxy * nxy, ncell = 3 * npsl;
    if (H.n_records < 0 || H.index_offset < (int64_t)sizeof(H) || H.data_offset % (int64_t)kAlign != 0 ||
        H.data_offset < H.index_offset + (ncell + 1) * 8)
        return set_arg_error("lsm_pslfile_run: corrupt PSL file header");
    struct stat sb;
    if (fstat(f.fd, &sb) != 0) return set_io_error("lsm_pslfile_run: stat", path, errno);
    if ((int64_t)sb.st_size < H.data_offset + H.n_records * 32)
        return set_arg_error("lsm_pslfile_run: PSL file shorter than its header says");
    std::vector<int64_t> cs((size_t)ncell + 1);
    if (!read_all(f.fd, cs.data(), cs.size() * 8, (off_t)H.index_offset))
        return set_io_error("lsm_pslfile_run: index", path, errno);
    if (cs[0] != 0 || cs[ncell] != H.n_records) return set_arg_error("lsm_pslfile_run: corrupt PSL file index");
    for (int64_t c = 0; c < ncell; ++c)
        if (cs[c + 1] < cs[c]) return set_arg_error("lsm_pslfile_run: corrupt PSL file index");

    // the field's cells (inclusion class 0 for primaries, 1 for scatter and
    // electrons) and its jaw opening on the upper jaw surfaces
    LSM_CUDA(cudaDeviceSynchronize());
    std::vector<uint8_t> incl((size_t)2 * npsl);
    float jaw[4];
    LSM_CUDA(cudaMemcpy(incl.data(), field->d_incl, incl.size(), cudaMemcpyDeviceToHost));
    LSM_CUDA(cudaMemcpy(jaw, field->d_jaws_f, sizeof(jaw), cudaMemcpyDeviceToHost));
    std::vector<std::pair<int64_t, int64_t>> ranges;
    int64_t N = 0;
    for (int s = 0; s < 3; ++s)
        for (int64_t j = 0; j < npsl; ++j) {
            const int64_t c = s * npsl + j;
            if (!incl[(size_t)((s ? 1 : 0) * npsl + j)] || cs[c + 1] == cs[c]) continue;
            if (!ranges.empty() && ranges.back().second == cs[c]) ranges.back().second = cs[c + 1];
            else ranges.emplace_back(cs[c], cs[c + 1]);
            N += cs[c + 1] - cs[c];
        }
    if (N == 0) return set_arg_error("lsm_pslfile_run: the field includes no record of the file");
    PslGeom G;
    for (int k = 0; k < 4; ++k) G.jaw[k] = jaw[k];
    G.zy_rel = field->sp.zy_rel; G.zx_rel = field->sp.zx_rel;
    G.z_rel = (float)(ph->z0 - field->z_phsp);
    G.x0 = (float)ph->x0; G.y0 = (float)ph->y0;

    const int64_t CH = opts->chunk > 0 ? std::min<int64_t>(opts->chunk, (int64_t)1 << 24) : ((int64_t)1 << 22);
    const size_t cbytes = (size_t)CH * sizeof(PslRec);
    int is_cold = 0;
    if (cold) {
        fdatasync(f.fd);
        is_cold = posix_fadvise(f.fd, 0, 0, POSIX_FADV_DONTNEED) == 0;
    }
    posix_fadvise(f.fd, 0, 0, POSIX_FADV_SEQUENTIAL);

    std::lock_guard<std::mutex> pool_lock(g_pool.m);
    lsm_status rc = g_pool.get(cbytes);
    if (rc) return rc;
    PslFileRun *R = nullptr;
    rc = pslfile_begin(ph, t, opts, CH, n_batches, seed, st, &R);
    if (rc) return rc;
    cudaStream_t cst = nullptr;
    cudaEvent_t h2d[3] = {}, c0[3] = {}, c1[3] = {}, comp[2] = {};
    auto make_events = [&]() -> cudaError_t {
        cudaError_t e = cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&h2d[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreate(&c0[k]);
            if (e == cudaSuccess) e = cudaEventCreate(&c1[k]);
        }
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&comp[k], cudaEventDisableTiming);
        return e;
    };
    cudaError_t ce = make_events();
    if (ce != cudaSuccess) rc = set_cuda_error(ce, "lsm_pslfile_run: stream/events");

    // reader thread: fills host buffer (c mod 3) with chunk c
    std::mutex m;
    std::condition_variable cv;
    bool filled[3] = {false, false, false}, stop = false;
    int read_err = 0;
    bool read_failed = false;
    Chunk desc[3];
    double t_read = 0.0;
    int64_t bytes = 0;
    const int fd = f.fd;
    const int64_t data_off = H.data_offset;
    bool reader_done = false;
    std::thread reader([&]() {
        int64_t c = 0;
        for (int p = 0; p < n_passes; ++p) {
            size_t r = 0;
            int64_t cur = ranges.empty() ? 0 : ranges[0].first, j = 0;
            while (j < N) {
                const int k = (int)(c % 3);
                {
                    std::unique_lock<std::mutex> lk(m);
                    cv.wait(lk, [&] { return !filled[k] || stop; });
                    if (stop) return;
                }
                char *buf = (char *)g_pool.h[k];
                int64_t got = 0;
                const double t0 = now_s();
                // the chunk's pieces of PSL ranges, then kReadThreads parallel
                // reads over equal shares of the chunk
                std::vector<Seg> segs;
                while (got < CH && j < N) {
                    const int64_t len = std::min(CH - got, ranges[r].second - cur);
                    segs.push_back({got, cur, len});
                    got += len; cur += len; j += len;
                    if (cur == ranges[r].second && ++r < ranges.size()) cur = ranges[r].first;
                }
                const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(kReadThreads, got * 32 / (8 << 20)));
                std::vector<int> errs((size_t)nt, 0);
                std::vector<std::thread> pool;
                for (int q = 1; q < nt; ++q)
                    pool.emplace_back([&, q] { errs[q] = read_share(fd, data_off, segs, buf, got * q / nt, got * (q + 1) / nt); });
                errs[0] = read_share(fd, data_off, segs, buf, 0, got / nt);
                for (auto &th : pool) th.join();
                for (int e : errs)
                    if (e) {
                        std::lock_guard<std::mutex> lk(m);
                        read_err = e;
                        read_failed = true;
                        reader_done = true;
                        cv.notify_all();
                        return;
                    }
                const double t1 = now_s();
                std::lock_guard<std::mutex> lk(m);
                t_read += t1 - t0;
                bytes += got * 32;
                desc[k].n = got;
                desc[k].i0 = j - got;
                desc[k].g0 = (uint64_t)p * (uint64_t)N + (uint64_t)(j - got);
                desc[k].end_of_pass = j == N;
                filled[k] = true;
                ++c;
                cv.notify_all();
            }
        }
        std::lock_guard<std::mutex> lk(m);
        reader_done = true;
        cv.notify_all();
    });

    double t_copy = 0.0;
    int64_t chunks = 0, records = 0;
    for (int64_t c = 0; rc == LSM_OK; ++c) {
        const int k = (int)(c % 3), db = (int)(c % 2);
        Chunk ck;
        {
            std::unique_lock<std::mutex> lk(m);
            cv.wait(lk, [&] { return filled[k] || reader_done; });
            if (!filled[k]) {
                if (read_failed) rc = set_io_error("lsm_pslfile_run: read", path, read_err);
                break;
            }
            ck = desc[k];
        }
        cudaError_t e = cudaSuccess;
        if (c >= 2) e = cudaStreamWaitEvent(cst, comp[db], 0);   // device buffer free again
        if (e == cudaSuccess) e = cudaEventRecord(c0[k], cst);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g_pool.d[db], g_pool.h[k], (size_t)ck.n * 32, cudaMemcpyHostToDevice, cst);
        if (e == cudaSuccess) e = cudaEventRecord(c1[k], cst);
        if (e == cudaSuccess) e = cudaEventRecord(h2d[k], cst);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h2d[k], 0);
        if (e != cudaSuccess) { rc = set_cuda_error(e, "lsm_pslfile_run: copy"); break; }
        rc = pslfile_chunk(R, g_pool.d[db], ck.n, ck.g0, ck.i0, G, st);
        if (rc) break;
        if ((e = cudaEventRecord(comp[db], st)) != cudaSuccess) { rc = set_cuda_error(e, "lsm_pslfile_run"); break; }
        if (ck.end_of_pass && (rc = pslfile_end_pass(R, st)) != LSM_OK) break;
        // the host buffer is free once its copy has landed
        if ((e = cudaEventSynchronize(c1[k])) != cudaSuccess) { rc = set_cuda_error(e, "lsm_pslfile_run: copy"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, c0[k], c1[k]);
        t_copy += 1e-3 * ms;
        ++chunks;
        records += ck.n;
        std::lock_guard<std::mutex> lk(m);
        filled[k] = false;
        cv.notify_all();
    }
    {
        std::lock_guard<std::mutex> lk(m);
        stop = true;
        cv.notify_all();
    }
    reader.join();
    cudaError_t se = cudaStreamSynchronize(st);
    if (cst) cudaStreamSynchronize(cst);
    const lsm_status rf = pslfile_finish(R, st);
    if (rc == LSM_OK && se != cudaSuccess) rc = set_cuda_error(se, "lsm_pslfile_run");
    if (rc == LSM_OK && records != (int64_t)n_passes * N) rc = set_io_error("lsm_pslfile_run: read", path, 0);
    if (rc == LSM_OK) rc = rf;
    for (int k = 0; k < 3; ++k) {
        if (h2d[k]) cudaEventDestroy(h2d[k]);
        if (c0[k]) cudaEventDestroy(c0[k]);
        if (c1[k]) cudaEventDestroy(c1[k]);
    }
    for (auto &e : comp) if (e) cudaEventDestroy(e);
    if (cst) cudaStreamDestroy(cst);
    if (stats) {
        stats->records = records;
        stats->bytes = bytes;
        stats->chunks = chunks;
        stats->t_read_s = t_read;
        stats->t_copy_s = t_copy;
        stats->t_total_s = now_s() - t_start;
        stats->dose_scale = (double)n_batches * H.w_record;
        stats->cold = is_cold;
        stats->pad = 0;
    }
    return rc;
}
