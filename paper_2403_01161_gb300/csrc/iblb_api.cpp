// iblb_api.cpp -- host side of the libiblb C ABI (include/iblb.h): workspace
// layout, mesh construction, the step schedule and the synchronising
// readouts.  All device work is launched through iblb_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "iblb_internal.h"

using iblb::Ctl;
using iblb::LbView;
using iblb::MeshView;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(IBL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t ctl = 0, frames = 0, frames_t = 0, f = 0, force = 0, vel = 0, rec = 0, ind = 0, total = 0;
};

long long pop_stride(long long nodes) { return (nodes + 63) / 64 * 64; }

bool lb_layout(const ibl_lb_params *p, int n_frames, Layout &L)
{
    if (!p || p->version != IBL_ABI_VERSION) return false;
    for (int a = 0; a < 3; ++a)
        if (p->n[a] < 4 || (p->bc[a] != IBL_BC_ZOU_HE && p->bc[a] != IBL_BC_PERIODIC)) return false;
    if (p->precision != IBL_FP32_DEV && p->precision != IBL_FP64) return false;
    if (n_frames < 1) return false;
    const long long nodes = (long long)p->n[0] * p->n[1] * p->n[2];
    if (19 * pop_stride(nodes) + 64 > 0x7fffffffLL) return false;  // 32-bit population indices
    const size_t es = p->precision == IBL_FP64 ? 8 : 4;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = align256(off + b);
        return o;
    };
    L.ctl = take(sizeof(Ctl));
    L.frames = take(sizeof(double) * 9 * (size_t)n_frames);
    L.frames_t = take(es * 9 * (size_t)n_frames);
    L.f = take(es * 19 * (size_t)pop_stride(nodes));
    L.force = take(es * 4 * (size_t)nodes);  // [nodes][4]: x, y, z, 0
    L.vel = take(es * 4 * (size_t)nodes);
    L.rec = p->record_fields ? take(es * 7 * (size_t)nodes) : 0;
    L.ind = take(((size_t)nodes + 3) / 4 * 4);  // inside flags, one byte per node
    L.total = off;
    return true;
}

struct MeshLayout {
    size_t r = 0, fn = 0, tris = 0, n2t_ptr = 0, n2t = 0, nb_ptr = 0, nb_idx = 0, s0 = 0, s1 = 0, s2 = 0,
           tm = 0, part = 0, cpart = 0, obs_part = 0, ring = 0, total = 0;
};

bool mesh_layout(int nv, int nt, MeshLayout &L)
{
    if (nv < 4 || nt < 4 || nv > (1 << 26) || nt > (1 << 26)) return false;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = align256(off + b);
        return o;
    };
    L.r = take(sizeof(double) * 3 * nv);
    L.fn = take(sizeof(double) * 3 * nv);
    L.tris = take(sizeof(int) * 3 * nt);
    L.n2t_ptr = take(sizeof(int) * (nv + 1));
    L.n2t = take(sizeof(int) * 3 * nt);
    L.nb_ptr = take(sizeof(int) * (nv + 1));
    L.nb_idx = take(sizeof(int) * 3 * nt);
    L.s0 = take(sizeof(double) * 3 * nv);
    L.s1 = take(sizeof(double) * 3 * nv);
    L.s2 = take(sizeof(double) * 3 * nv);
    L.tm = take(sizeof(double) * 3 * nt);
    L.part = take(sizeof(double) * 6 * (((size_t)nv + 7) / 8 + 1));  // one row per interpolation block
    L.cpart = take(sizeof(double) * 4 * iblb::kCentreBlocks);
    L.obs_part = take(sizeof(double) * 11 * iblb::kObsBlocksMax);
    L.ring = take(sizeof(ibl_observables) * iblb::kRingCap);
    L.total = off;
    return true;
}

enum { PROF_LB = 0, PROF_SPREAD = 1, PROF_INTERP = 2 };

struct Profiler {
    int mask = 0;
    int every = 1;        // bracket one launch in `every`
    long long seen[3] = {0, 0, 0};
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, int>> marks;  // (kind, first event index)
    size_t used = 0;
    static constexpr size_t kMax = 65536;

    cudaEvent_t take()
    {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void clear()
    {
        used = 0;
        marks.clear();
        seen[0] = seen[1] = seen[2] = 0;
    }
    ~Profiler()
    {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

}  // namespace

int iblb::iblb_set_error(int code, const char *msg) { return fail(code, msg); }

namespace {
// NVTX range over a C-ABI call, so that a profiler's timeline shows which
// library call issued which kernels (header-only NVTX: no cost unless a tool
// is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
};
}  // namespace

struct ibl_lb {
    ibl_lb_params p;
    LbView v;
    Layout lay;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    long long host_step = 0;
    bool recorded = false;
    ibl_mesh *mesh = nullptr;
    Profiler prof;
    // CUDA-graph replay of whole chunks of steps
    bool graphs = true;
    int chunk = 0;                       // chunk length of the schedule the graphs belong to (0 = none captured)
    // one graph per position in the schedule period when that period is the
    // bare 6 (AA parity x three patch buffers), else only slot 0
    static constexpr int kPhases = 6;
    cudaGraphExec_t gexec[kPhases] = {};
    // graphs of the shorter runs of steps around whole chunks (segments),
    // keyed by length and by the start's position in the schedule period;
    // captured by ibl_prepare_steps, or at a segment's second occurrence
    // (seen[] remembers the last kSeen segments run eagerly); the least
    // recently used graph is dropped first
    struct Segment {
        long long phase = -1, len = 0, used = 0;
        cudaGraphExec_t g = nullptr;
    };
    static constexpr int kSegments = 32, kSeen = 64;
    static constexpr long long kMaxSegment = 2048;
    Segment seg[kSegments];
    long long seg_clock = 0;
    long long seen[kSeen][2] = {};
    int seen_next = 0;
    long long steps_eager = 0, steps_replayed = 0;  // counts of ibl_step's two paths
    cudaStream_t cap_stream = nullptr;   // private streams used only for capture
    cudaStream_t cap_helper = nullptr;
    bool capturing = false;
    // With a droplet, a step runs on two streams: the bound stream carries the
    // lattice update of the nodes outside the droplet patch, the high-priority
    // helper stream the droplet kernels and the patch nodes.  evNear[p] marks
    // the end of the patch-node update (or of a regularisation) of the last
    // step of parity p, evFar[p] the end of the outside update and step count.
    cudaStream_t helper = nullptr;
    int hi_prio = 0;  // priority of the helper-stream kernels
    cudaEvent_t evNear[2] = {nullptr, nullptr}, evFar[2] = {nullptr, nullptr};
    cudaEvent_t evFork = nullptr, evJoin = nullptr;
    cudaEvent_t evCentre = nullptr;  // re-centring: the force kernel of the step has written the centre
    // a separate set for graph capture (events recorded inside a capture
    // cannot be waited on by eager launches)
    cudaEvent_t cNear[2] = {nullptr, nullptr}, cFar[2] = {nullptr, nullptr};
    cudaEvent_t cFork = nullptr, cJoin = nullptr, cCentre = nullptr;
    ~ibl_lb()
    {
        for (cudaGraphExec_t g : gexec)
            if (g) cudaGraphExecDestroy(g);
        for (Segment &sg : seg)
            if (sg.g) cudaGraphExecDestroy(sg.g);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (cap_helper) cudaStreamDestroy(cap_helper);
        if (helper) cudaStreamDestroy(helper);
        for (int k = 0; k < 2; ++k) {
            if (evNear[k]) cudaEventDestroy(evNear[k]);
            if (evFar[k]) cudaEventDestroy(evFar[k]);
            if (cNear[k]) cudaEventDestroy(cNear[k]);
            if (cFar[k]) cudaEventDestroy(cFar[k]);
        }
        if (evFork) cudaEventDestroy(evFork);
        if (evJoin) cudaEventDestroy(evJoin);
        if (cFork) cudaEventDestroy(cFork);
        if (cJoin) cudaEventDestroy(cJoin);
        if (evCentre) cudaEventDestroy(evCentre);
        if (cCentre) cudaEventDestroy(cCentre);
    }
};

struct ibl_mesh {
    ibl_lb *lb = nullptr;
    MeshView v;
    MeshLayout lay;
    std::vector<int> tris, nb_ptr, nb_idx;
    iblb::RegParams reg{0.1, 0.51, 0.01, 100, 1};
    int reg_every = 0;
    int readout_every = 0;
};

namespace {

void drop_graph(ibl_lb *lb);

int lb_status_from_device(ibl_lb *lb)
{
    Ctl c;
    cudaError_t e = cudaMemcpyAsync(&c, lb->ws + lb->lay.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "read control block");
    e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (c.err & IBL_ERRBIT_UNSTABLE) return fail(IBL_EUNSTABLE, "NaN density or |u| > 0.3 on some lattice node");
    if (c.err & IBL_ERRBIT_WALL)
        return fail(IBL_EWALL, "a droplet node's stencil reached a wet boundary node (or its position is invalid)");
    if (c.err & IBL_ERRBIT_NOCONV) return fail(IBL_ENOCONV, "mesh regularisation did not converge within max_iter");
    if (c.err & IBL_ERRBIT_TIMEOUT)
        return fail(IBL_ETIMEOUT, "the staged lattice update gave up waiting for its copies into shared memory");
    return IBL_OK;
}

// Returns the index of the end event to record after the launch, or -1.
int prof_begin(ibl_lb *lb, int kind, cudaStream_t s)
{
    if (!((lb->prof.mask >> kind) & 1) || lb->prof.marks.size() >= Profiler::kMax) return -1;
    if ((lb->prof.mask & 8) && !lb->capturing) return -1;  // graph replays only
    if (lb->prof.seen[kind]++ % lb->prof.every != 0) return -1;
    cudaEvent_t a = lb->prof.take();
    cudaEvent_t b = lb->prof.take();
    if (!a || !b) return -1;
    const int idx = (int)lb->prof.used - 2;
    lb->prof.marks.push_back({kind, idx});
    // inside a capture the record must become a graph node of its own
    if (lb->capturing) cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
    else cudaEventRecord(a, s);
    return idx + 1;
}

void prof_end(ibl_lb *lb, int end_idx, cudaStream_t s)
{
    if (end_idx < 0) return;
    if (lb->capturing) cudaEventRecordWithFlags(lb->prof.pool[end_idx], s, cudaEventRecordExternal);
    else cudaEventRecord(lb->prof.pool[end_idx], s);
}

// One step.  sL: the bound stream (or the capture stream), sH: the helper
// stream (or its capture twin).  Without a droplet everything runs on sL.
int one_step(ibl_lb *lb, bool record, cudaStream_t sL, cudaStream_t sH)
{
    cudaError_t e;
    ibl_mesh *m = lb->mesh;
    const int par = (int)(lb->host_step & 1);
    const bool odd = par != 0;
    const long long next = lb->host_step + 1;
    const int pbuf = (int)(lb->host_step % 3), pnext = (int)(next % 3);
    cudaEvent_t *evNear = lb->capturing ? lb->cNear : lb->evNear;
    cudaEvent_t *evFar = lb->capturing ? lb->cFar : lb->evFar;
    if (!m) {
        const int pl = prof_begin(lb, PROF_LB, sL);
        e = iblb::launch_lattice(lb->v, odd, record, iblb::LAUNCH_FULL, pbuf, sL);
        prof_end(lb, pl, sL);
        if (e != cudaSuccess) return cuda_fail(e, "lattice launch");
        lb->host_step = next;
        return IBL_OK;
    }
    // helper stream: forces + spread (and the next step's patch), then the
    // patch nodes once the previous outside update has finished
    // with re-centring, first the step's centre (from the positions the
    // previous step left), which the outside update reads on its faces
    cudaEvent_t evCentre = lb->capturing ? lb->cCentre : lb->evCentre;
    e = cudaSuccess;
    if (lb->v.recentre) {
        e = iblb::launch_centre(lb->v, m->v, pbuf, sH, lb->hi_prio);
        if (e == cudaSuccess) e = cudaEventRecord(evCentre, sH);
    }
    // with a viscosity ratio, the inside flags of this step's patch nodes
    // (read and cleared by the patch update below)
    if (e == cudaSuccess && lb->v.visc) e = iblb::launch_indicator(lb->v, m->v, pbuf, sH, lb->hi_prio);
    const int ps = prof_begin(lb, PROF_SPREAD, sH);
    if (e == cudaSuccess) e = iblb::launch_spread(lb->v, m->v, pnext, sH, lb->hi_prio);
    prof_end(lb, ps, sH);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sH, evFar[par ^ 1], 0);
    if (e == cudaSuccess) e = iblb::launch_near(lb->v, odd, record, pbuf, sH, lb->hi_prio);
    if (e == cudaSuccess) e = cudaEventRecord(evNear[par], sH);
    if (e != cudaSuccess) return cuda_fail(e, "droplet-side launch");
    // bound stream: the outside nodes once the previous patch update (and
    // regularisation) has finished; one thread of that kernel closes the step
    // (step counter, frame of the next step)
    e = cudaStreamWaitEvent(sL, evNear[par ^ 1], 0);
    if (e == cudaSuccess && lb->v.recentre) e = cudaStreamWaitEvent(sL, evCentre, 0);
    const int pl = prof_begin(lb, PROF_LB, sL);
    if (e == cudaSuccess) e = iblb::launch_lattice(lb->v, odd, record, iblb::LAUNCH_FAR, pbuf, sL);
    prof_end(lb, pl, sL);
    if (e == cudaSuccess) e = cudaEventRecord(evFar[par], sL);
    if (e != cudaSuccess) return cuda_fail(e, "lattice launch");
    // helper stream: interpolation + advection, scheduled regularisation
    // (which rewrites the next step's patch, so the next outside update
    // waits for it) and shape record (which reads the step counter)
    const int pi = prof_begin(lb, PROF_INTERP, sH);
    e = iblb::launch_interp(lb->v, m->v, sH, lb->hi_prio);
    prof_end(lb, pi, sH);
    if (e != cudaSuccess) return cuda_fail(e, "interpolation launch");
    if (m->reg_every > 0 && next % m->reg_every == 0) {
        e = iblb::launch_regularize(lb->v, m->v, m->reg, pnext, sH, lb->hi_prio);
        if (e == cudaSuccess) e = cudaEventRecord(evNear[par], sH);
        if (e != cudaSuccess) return cuda_fail(e, "regularisation launch");
    }
    if (m->readout_every > 0 && next % m->readout_every == 0) {
        // the record reads the step counter: after this step's count, and
        // before the next step's (the next outside update waits for it)
        e = cudaStreamWaitEvent(sH, evFar[par], 0);
        if (e == cudaSuccess) e = iblb::launch_observables(lb->v, m->v, sH, lb->hi_prio);
        if (e == cudaSuccess) e = cudaEventRecord(evNear[par], sH);
        if (e != cudaSuccess) return cuda_fail(e, "observables launch");
    }
    lb->host_step = next;
    return IBL_OK;
}

// Orders `to` after everything enqueued so far on `from`.
cudaError_t join(cudaStream_t from, cudaStream_t to, cudaEvent_t ev)
{
    cudaError_t e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
    return e;
}

// ---- mesh construction (library's own implementation) ---------------------
void unit(double v[3])
{
    const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n;
    v[1] /= n;
    v[2] /= n;
}

// Subdivided icosahedron: base vertices (+-1, +-p, 0) cyclically in the
// order below, base faces = mutually adjacent triples sorted ascending and
// oriented outward; each level splits every face into four through the edge
// midpoints (created on first use, projected to the unit sphere).
void icosphere(int level, std::vector<double> &xyz, std::vector<int> &tri)
{
    const double p = (1.0 + std::sqrt(5.0)) / 2.0;
    const double raw[12][3] = {{-1, p, 0}, {1, p, 0}, {-1, -p, 0}, {1, -p, 0}, {0, -1, p}, {0, 1, p},
                               {0, -1, -p}, {0, 1, -p}, {p, 0, -1}, {p, 0, 1}, {-p, 0, -1}, {-p, 0, 1}};
    auto dist = [&](int a, int b) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += (raw[a][k] - raw[b][k]) * (raw[a][k] - raw[b][k]);
        return std::sqrt(s);
    };
    tri.clear();
    for (int a = 0; a < 12; ++a)
        for (int b = a + 1; b < 12; ++b)
            for (int c = b + 1; c < 12; ++c) {
                if (std::fabs(dist(a, b) - 2) > 1e-9 || std::fabs(dist(b, c) - 2) > 1e-9 ||
                    std::fabs(dist(c, a) - 2) > 1e-9)
                    continue;
                double e1[3], e2[3], n[3];
                for (int k = 0; k < 3; ++k) {
                    e1[k] = raw[b][k] - raw[a][k];
                    e2[k] = raw[c][k] - raw[a][k];
                }
                n[0] = e1[1] * e2[2] - e1[2] * e2[1];
                n[1] = e1[2] * e2[0] - e1[0] * e2[2];
                n[2] = e1[0] * e2[1] - e1[1] * e2[0];
                const double out = n[0] * (raw[a][0] + raw[b][0] + raw[c][0]) +
                                   n[1] * (raw[a][1] + raw[b][1] + raw[c][1]) +
                                   n[2] * (raw[a][2] + raw[b][2] + raw[c][2]);
                if (out > 0) tri.insert(tri.end(), {a, b, c});
                else tri.insert(tri.end(), {a, c, b});
            }
    xyz.clear();
    for (int i = 0; i < 12; ++i) {
        double v[3] = {raw[i][0], raw[i][1], raw[i][2]};
        unit(v);
        xyz.insert(xyz.end(), {v[0], v[1], v[2]});
    }
    for (int l = 0; l < level; ++l) {
        std::map<std::pair<int, int>, int> mid;
        std::vector<int> nt;
        nt.reserve(tri.size() * 4);
        auto midpoint = [&](int i, int j) {
            const auto key = std::make_pair(std::min(i, j), std::max(i, j));
            auto it = mid.find(key);
            if (it != mid.end()) return it->second;
            const int id = (int)(xyz.size() / 3);
            double v[3] = {(xyz[3 * i] + xyz[3 * j]) * 0.5, (xyz[3 * i + 1] + xyz[3 * j + 1]) * 0.5,
                           (xyz[3 * i + 2] + xyz[3 * j + 2]) * 0.5};
            unit(v);
            xyz.insert(xyz.end(), {v[0], v[1], v[2]});
            mid[key] = id;
            return id;
        };
        for (size_t t = 0; t < tri.size(); t += 3) {
            const int a = tri[t], b = tri[t + 1], c = tri[t + 2];
            const int mab = midpoint(a, b);
            const int mbc = midpoint(b, c);
            const int mca = midpoint(c, a);
            nt.insert(nt.end(), {a, mab, mca, b, mbc, mab, c, mca, mbc, mab, mbc, mca});
        }
        tri.swap(nt);
    }
}

// Closed, consistently oriented 2-manifold: every directed edge once and its
// reverse once.  Builds one-ring neighbour CSR (ascending) and node-to-
// triangle CSR (entries 3*t + slot, in triangle order).
bool build_topology(int nv, const std::vector<int> &tri, std::vector<int> &nb_ptr, std::vector<int> &nb_idx,
                    std::vector<int> &n2t_ptr, std::vector<int> &n2t, std::string &why)
{
    const int nt = (int)(tri.size() / 3);
    std::vector<std::pair<int, int>> de;
    de.reserve(3 * nt);
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3];
            if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) {
                why = "triangle index out of range or degenerate";
                return false;
            }
            de.push_back({a, b});
        }
    std::vector<std::pair<int, int>> sorted = de;
    std::sort(sorted.begin(), sorted.end());
    for (size_t k = 1; k < sorted.size(); ++k)
        if (sorted[k] == sorted[k - 1]) {
            why = "directed edge used twice (inconsistent orientation or non-manifold)";
            return false;
        }
    for (auto &e : de)
        if (!std::binary_search(sorted.begin(), sorted.end(), std::make_pair(e.second, e.first))) {
            why = "mesh is not closed";
            return false;
        }
    std::vector<std::vector<int>> nb(nv);
    for (auto &e : de) nb[e.first].push_back(e.second);
    nb_ptr.assign(nv + 1, 0);
    nb_idx.clear();
    for (int i = 0; i < nv; ++i) {
        std::sort(nb[i].begin(), nb[i].end());
        if (nb[i].empty()) {
            why = "node without triangles";
            return false;
        }
        nb_ptr[i + 1] = nb_ptr[i] + (int)nb[i].size();
        nb_idx.insert(nb_idx.end(), nb[i].begin(), nb[i].end());
    }
    std::vector<std::vector<int>> inc(nv);
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) inc[tri[3 * t + k]].push_back(3 * t + k);
    n2t_ptr.assign(nv + 1, 0);
    n2t.clear();
    for (int i = 0; i < nv; ++i) {
        n2t_ptr[i + 1] = n2t_ptr[i] + (int)inc[i].size();
        n2t.insert(n2t.end(), inc[i].begin(), inc[i].end());
    }
    return true;
}

// Whether the outside update keeps its L2 prefetch beside a droplet whose
// nodes start at r: only while the droplet's patch (its bounding box grown
// by the stencil reach and one node of motion, floor(min) - 2 ..
// floor(max) + 3 per axis, as the device writes it) has at most 150k nodes.  The patch's populations and 4-wide force and velocity
// records, about 108 B a node in FP32, are kept in L2 for the droplet
// kernels; a larger patch leaves too little room for lines fetched a wave
// early.  Measured with the prefetch on and off: 128^3 droplet (patch 27k
// nodes) 57.7 against 58.9 us, 256^3 droplet (157k nodes at the start,
// growing as it deforms) 436.6 against 425.6 us.
bool prefetch_with_patch(const double *r, int nv)
{
    double lo[3] = {r[0], r[1], r[2]}, hi[3] = {r[0], r[1], r[2]};
    for (int i = 1; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], r[3 * i + a]);
            hi[a] = std::max(hi[a], r[3 * i + a]);
        }
    double nodes = 1.0;
    for (int a = 0; a < 3; ++a) nodes *= std::floor(hi[a]) - std::floor(lo[a]) + 6.0;
    return nodes <= 150000.0;
}

int mesh_attach(ibl_lb *lb, int nv, const double *r, int nt, const int *tri_in, double sigma, void *ws,
                size_t bytes, ibl_mesh **out)
{
    if (!lb || !r || !tri_in || !out) return fail(IBL_EINVAL, "null argument");
    if (lb->mesh) return fail(IBL_EINVAL, "the lattice already carries a droplet");
    MeshLayout L;
    if (!mesh_layout(nv, nt, L)) return fail(IBL_EINVAL, "bad mesh size");
    if (!ws || bytes < L.total) return fail(IBL_ENOMEM, "mesh workspace too small");
    if (((uintptr_t)ws & 255) != 0) return fail(IBL_EINVAL, "workspace must be 256-byte aligned");
    if (!(sigma >= 0) || !std::isfinite(sigma)) return fail(IBL_EINVAL, "sigma must be finite and >= 0");
    std::vector<int> tri(tri_in, tri_in + 3 * (size_t)nt);
    std::vector<int> nb_ptr, nb_idx, n2t_ptr, n2t;
    std::string why;
    if (!build_topology(nv, tri, nb_ptr, nb_idx, n2t_ptr, n2t, why)) return fail(IBL_EINVAL, "mesh: " + why);
    if ((int)nb_idx.size() != 3 * nt) return fail(IBL_EINVAL, "mesh: unexpected neighbour count");
    for (int i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(r[i])) return fail(IBL_EINVAL, "mesh: non-finite position");
    ibl_mesh *m = new ibl_mesh();
    m->lb = lb;
    m->lay = L;
    char *w = static_cast<char *>(ws);
    m->v.nv = nv;
    m->v.nt = nt;
    m->v.sigma = sigma;
    m->v.r = reinterpret_cast<double *>(w + L.r);
    m->v.fn = reinterpret_cast<double *>(w + L.fn);
    m->v.tris = reinterpret_cast<const int *>(w + L.tris);
    m->v.n2t_ptr = reinterpret_cast<const int *>(w + L.n2t_ptr);
    m->v.n2t = reinterpret_cast<const int *>(w + L.n2t);
    m->v.nb_ptr = reinterpret_cast<const int *>(w + L.nb_ptr);
    m->v.nb_idx = reinterpret_cast<const int *>(w + L.nb_idx);
    m->v.s0 = reinterpret_cast<double *>(w + L.s0);
    m->v.s1 = reinterpret_cast<double *>(w + L.s1);
    m->v.s2 = reinterpret_cast<double *>(w + L.s2);
    m->v.tm = reinterpret_cast<double *>(w + L.tm);
    m->v.part = reinterpret_cast<double *>(w + L.part);
    m->v.cpart = reinterpret_cast<double *>(w + L.cpart);
    m->v.obs_part = reinterpret_cast<double *>(w + L.obs_part);
    m->v.ring = reinterpret_cast<ibl_observables *>(w + L.ring);
    m->v.ring_cap = iblb::kRingCap;
    m->tris = tri;
    m->nb_ptr = nb_ptr;
    m->nb_idx = nb_idx;
    cudaStream_t s = lb->stream;
    cudaError_t e = cudaSuccess;
    auto up = [&](size_t off, const void *src, size_t n) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(w + off, src, n, cudaMemcpyHostToDevice, s);
    };
    up(L.r, r, sizeof(double) * 3 * nv);
    up(L.tris, tri.data(), sizeof(int) * 3 * nt);
    up(L.n2t_ptr, n2t_ptr.data(), sizeof(int) * (nv + 1));
    up(L.n2t, n2t.data(), sizeof(int) * n2t.size());
    up(L.nb_ptr, nb_ptr.data(), sizeof(int) * (nv + 1));
    up(L.nb_idx, nb_idx.data(), sizeof(int) * nb_idx.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(w + L.fn, 0, sizeof(double) * 3 * nv, s);
    if (e == cudaSuccess) e = iblb::launch_patch_from_mesh(lb->v, m->v, (int)(lb->host_step % 3), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors above are pageable temporaries
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "mesh upload");
    }
    drop_graph(lb);
    lb->mesh = m;
    lb->v.prefetch = prefetch_with_patch(r, nv) ? 1 : 0;
    *out = m;
    return IBL_OK;
}

}  // namespace

namespace {

void drop_graph(ibl_lb *lb)
{
    if (!lb) return;
    for (cudaGraphExec_t &g : lb->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (ibl_lb::Segment &sg : lb->seg) {
        if (sg.g) cudaGraphExecDestroy(sg.g);
        sg = ibl_lb::Segment{};
    }
    for (auto &k : lb->seen) k[0] = k[1] = 0;
    lb->chunk = 0;
}

long long gcd_ll(long long a, long long b) { return b == 0 ? a : gcd_ll(b, a % b); }

// Schedule period: the launches of a step repeat with this period in the
// step index -- 6 (AA parity and the three patch buffers), times the
// regularisation and readout periods.
long long schedule_period(const ibl_lb *lb)
{
    long long c = 6;
    const ibl_mesh *m = lb->mesh;
    auto lcm = [&](long long a, long long b) { return a / gcd_ll(a, b) * b; };
    if (m && m->reg_every > 0) c = lcm(c, m->reg_every);
    if (m && m->readout_every > 0) c = lcm(c, m->readout_every);
    return c;
}

// Steps per chunk: a multiple of the schedule period, at least 32; 0 when
// that would exceed 2048.
int chunk_length(const ibl_lb *lb)
{
    long long c = schedule_period(lb);
    if (c > 2048) return 0;
    while (c < 32) c *= 2;
    return (int)c;
}

// Creates the helper stream (highest priority) and the step events.
int ensure_streams(ibl_lb *lb)
{
    if (lb->helper) return IBL_OK;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    lb->hi_prio = hi;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&lb->helper, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&lb->cap_stream, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&lb->cap_helper, cudaStreamNonBlocking, hi);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&lb->evNear[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->evFar[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->cNear[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->cFar[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->evFork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->evJoin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->cFork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->cJoin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->evCentre, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lb->cCentre, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "stream/event creation");
    return IBL_OK;
}

// Captures n steps from host_step into *out: fork the helper capture stream
// off the main one, re-record the step events inside the capture, run the
// steps (hook(k, main, helper) first enqueues whatever step k needs before
// it), join back.  host_step is left unchanged.
template <typename Hook>
int capture_steps(ibl_lb *lb, int n, bool record, Hook &&hook, cudaGraphExec_t *out)
{
    int st = ensure_streams(lb);
    if (st != IBL_OK) return st;
    const long long saved = lb->host_step;
    cudaStream_t cL = lb->cap_stream, cH = lb->cap_helper;
    cudaError_t e = cudaStreamBeginCapture(cL, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    lb->capturing = true;
    e = join(cL, cH, lb->cFork);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(lb->cNear[k], cH);
        if (e == cudaSuccess) e = cudaEventRecord(lb->cFar[k], cL);
    }
    if (e != cudaSuccess) st = cuda_fail(e, "capture fork");
    for (int k = 0; k < n && st == IBL_OK; ++k) {
        st = hook(k, cL, cH);
        if (st == IBL_OK) st = one_step(lb, record, cL, cH);
    }
    if (st == IBL_OK) {
        e = join(cH, cL, lb->cJoin);
        if (e != cudaSuccess) st = cuda_fail(e, "capture join");
    }
    lb->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cL, &g);
    if (e2 != cudaSuccess && st == IBL_OK) st = cuda_fail(e2, "end capture");
    if (st == IBL_OK) {
        const cudaError_t e3 = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
        if (e3 != cudaSuccess) st = cuda_fail(e3, "graph instantiate");
    }
    if (g) cudaGraphDestroy(g);
    lb->host_step = saved;
    return st;
}

// Captures one chunk of plain steps starting at the current step into
// graph slot `slot`.
int capture_chunk(ibl_lb *lb, int chunk, int slot)
{
    const int st =
        capture_steps(lb, chunk, false, [](int, cudaStream_t, cudaStream_t) { return IBL_OK; }, &lb->gexec[slot]);
    if (st == IBL_OK) lb->chunk = chunk;
    else drop_graph(lb);
    return st;
}

// A run of steps as ibl_step executes it: a whole chunk (graph slot `slot`)
// or a segment of `len` steps (graph keyed by `phase`, else eager).
struct Piece {
    bool chunk;
    int slot;
    long long start, len, phase;
};

// Splits n steps from the current step into whole chunks -- at chunk
// boundaries, or at any step when the schedule period is the bare 6 (one
// graph per phase) -- and the segments between them (at most kMaxSegment
// steps each).
void plan_steps(const ibl_lb *lb, long long n, std::vector<Piece> &out)
{
    out.clear();
    const int chunk = lb->graphs ? chunk_length(lb) : 0;
    const long long period = schedule_period(lb);
    const bool keyed = chunk > 0 && period <= ibl_lb::kPhases;
    long long s = lb->host_step, done = 0;
    while (done < n) {
        if (chunk > 0 && n - done >= chunk && (keyed || s % chunk == 0)) {
            out.push_back({true, keyed ? (int)(s % period) : 0, s, chunk, s % period});
            s += chunk;
            done += chunk;
            continue;
        }
        long long len = n - done;
        if (chunk > 0 && !keyed) {
            const long long to_boundary = (chunk - s % chunk) % chunk;
            if (n - done - to_boundary >= chunk) len = to_boundary;
        }
        len = std::min(len, ibl_lb::kMaxSegment);
        out.push_back({false, 0, s, len, s % period});
        s += len;
        done += len;
    }
}

ibl_lb::Segment *find_segment(ibl_lb *lb, long long phase, long long len)
{
    for (ibl_lb::Segment &sg : lb->seg)
        if (sg.g && sg.phase == phase && sg.len == len) {
            sg.used = ++lb->seg_clock;
            return &sg;
        }
    return nullptr;
}

// Whether the segment (phase, len) ran eagerly before (since the graphs were
// last dropped); records it if not.
bool seen_before(ibl_lb *lb, long long phase, long long len)
{
    for (const auto &k : lb->seen)
        if (k[1] == len && k[0] == phase) return true;
    lb->seen[lb->seen_next][0] = phase;
    lb->seen[lb->seen_next][1] = len;
    lb->seen_next = (lb->seen_next + 1) % ibl_lb::kSeen;
    return false;
}

// Captures the segment piece `pc` into the least recently used slot and
// uploads it to the device (its first launch then costs no more than the
// next ones).
int capture_segment(ibl_lb *lb, const Piece &pc, ibl_lb::Segment **out)
{
    ibl_lb::Segment *slot = &lb->seg[0];
    for (ibl_lb::Segment &sg : lb->seg) {
        if (!sg.g) {
            slot = &sg;
            break;
        }
        if (sg.used < slot->used) slot = &sg;
    }
    if (slot->g) cudaGraphExecDestroy(slot->g);
    *slot = ibl_lb::Segment{};
    const long long saved = lb->host_step;
    lb->host_step = pc.start;
    const int st = capture_steps(lb, (int)pc.len, false, [](int, cudaStream_t, cudaStream_t) { return IBL_OK; },
                                 &slot->g);
    lb->host_step = saved;
    if (st != IBL_OK) {
        slot->g = nullptr;
        return st;
    }
    const cudaError_t e = cudaGraphUpload(slot->g, lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph upload");
    slot->phase = pc.phase;
    slot->len = pc.len;
    slot->used = ++lb->seg_clock;
    lb->chunk = chunk_length(lb);  // the schedule the graphs belong to
    *out = slot;
    return IBL_OK;
}

}  // namespace

struct ibl_ensemble {
    std::vector<ibl_lb *> m;
    iblb::EnsembleView v{};
    cudaStream_t stream = nullptr;       // the members' bound stream
    cudaStream_t helper = nullptr;       // high-priority helper stream (droplet kernels, patch nodes)
    int hi_prio = 0;
    cudaStream_t cap_stream = nullptr, cap_helper = nullptr;  // capture twins
    cudaGraphExec_t gexec = nullptr;     // whole chunk
    int chunk = 0;
    bool capturing = false;
    // step events as in ibl_lb: evNear[p] the end of the patch update (and
    // regularisations, shape records) of the last step of parity p, evFar[p]
    // the end of its outside update; a second set for use inside captures
    cudaEvent_t evNear[2] = {nullptr, nullptr}, evFar[2] = {nullptr, nullptr};
    cudaEvent_t cNear[2] = {nullptr, nullptr}, cFar[2] = {nullptr, nullptr};
    cudaEvent_t evFork = nullptr, evJoin = nullptr, evCentre = nullptr;
    cudaEvent_t cFork = nullptr, cJoin = nullptr, cCentre = nullptr;
    ~ibl_ensemble()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (cap_helper) cudaStreamDestroy(cap_helper);
        if (helper) cudaStreamDestroy(helper);
        for (cudaEvent_t ev : {evNear[0], evNear[1], evFar[0], evFar[1], cNear[0], cNear[1], cFar[0], cFar[1], evFork,
                               evJoin, evCentre, cFork, cJoin, cCentre})
            if (ev) cudaEventDestroy(ev);
    }
};

namespace {

struct EnsembleLayout {
    size_t lat_member[2] = {0, 0}, lat_start[2] = {0, 0}, node_member = 0, node_start = 0, total = 0;
    int lat_blocks[2] = {0, 0}, node_blocks = 0;
};

// Blocks of the batched lattice update of one member with nt threads per
// block: whole blocks per z plane.
long long lattice_blocks(const ibl_lb *lb, int nt)
{
    const long long nxy = (long long)lb->v.n[0] * lb->v.n[1];
    return (nxy + nt - 1) / nt * lb->v.n[2];
}

int ensemble_layout(int n, ibl_lb *const *members, EnsembleLayout &L, std::string &why)
{
    if (n < 1 || !members) {
        why = "need at least one member";
        return IBL_EINVAL;
    }
    long long lat[2] = {0, 0}, node = 0;
    for (int k = 0; k < n; ++k) {
        const ibl_lb *lb = members[k];
        if (!lb || !lb->mesh) {
            why = "every member needs a lattice with a droplet mesh";
            return IBL_EINVAL;
        }
        if ((long long)lb->v.n[0] * lb->v.n[1] >= (1LL << 22)) {
            why = "an ensemble member's z plane exceeds 2^22 nodes";
            return IBL_EINVAL;
        }
        lat[0] += lattice_blocks(lb, 128);
        lat[1] += lattice_blocks(lb, 256);
        node += ((long long)lb->mesh->v.nv + iblb::kFwdNodesPerBlock - 1) / iblb::kFwdNodesPerBlock;
    }
    if (lat[0] > 0x7fffffffLL) {
        why = "ensemble too large";
        return IBL_EINVAL;
    }
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = align256(off + b);
        return o;
    };
    for (int t = 0; t < 2; ++t) {
        L.lat_member[t] = take(sizeof(int) * lat[t]);
        L.lat_start[t] = take(sizeof(int) * (n + 1));
        L.lat_blocks[t] = (int)lat[t];
    }
    L.node_member = take(sizeof(int) * node);
    L.node_start = take(sizeof(int) * (n + 1));
    L.total = off;
    L.node_blocks = (int)node;
    return IBL_OK;
}

int ensemble_chunk(const ibl_ensemble *e)
{
    long long c = 6;
    auto lcm = [&](long long a, long long b) { return a / gcd_ll(a, b) * b; };
    for (ibl_lb *lb : e->m) {
        if (lb->mesh->reg_every > 0) c = lcm(c, lb->mesh->reg_every);
        if (lb->mesh->readout_every > 0) c = lcm(c, lb->mesh->readout_every);
        if (c > 2048) return 0;
    }
    while (c < 32) c *= 2;
    return (int)c;
}

int ensemble_streams(ibl_ensemble *en)
{
    if (en->helper) return IBL_OK;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    en->hi_prio = hi;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&en->helper, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&en->cap_stream, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&en->cap_helper, cudaStreamNonBlocking, hi);
    cudaEvent_t *evs[] = {&en->evNear[0], &en->evNear[1], &en->evFar[0], &en->evFar[1], &en->cNear[0], &en->cNear[1],
                          &en->cFar[0], &en->cFar[1], &en->evFork, &en->evJoin, &en->evCentre, &en->cFork,
                          &en->cJoin, &en->cCentre};
    for (cudaEvent_t *ev : evs)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "ensemble stream/event creation");
    return IBL_OK;
}

// One ensemble step on two streams, as one_step for a single droplet: on
// the helper stream sH the droplet kernels of every member (re-centring,
// triangle moments, forces + spread), the patch nodes once the previous
// outside update has finished, the interpolation, then each member's
// scheduled regularisation and shape record; on the bound stream sL the
// nodes outside every member's patch once the previous patch update has
// finished (its first block per member closes that member's step).
int ensemble_one_step(ibl_ensemble *e, cudaStream_t sL, cudaStream_t sH)
{
    const long long step = e->m[0]->host_step;
    const int par = (int)(step & 1);
    const long long next = step + 1;
    cudaEvent_t *evNear = e->capturing ? e->cNear : e->evNear;
    cudaEvent_t *evFar = e->capturing ? e->cFar : e->evFar;
    cudaEvent_t evCentre = e->capturing ? e->cCentre : e->evCentre;
    bool recentre = false;
    for (ibl_lb *lb : e->m) recentre = recentre || lb->v.recentre != 0;
    cudaError_t err = iblb::launch_ensemble_pre(e->v, step, sH, e->hi_prio);
    if (err == cudaSuccess && recentre) err = cudaEventRecord(evCentre, sH);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(sH, evFar[par ^ 1], 0);
    if (err == cudaSuccess) err = iblb::launch_ensemble_near(e->v, step, sH, e->hi_prio);
    if (err == cudaSuccess) err = cudaEventRecord(evNear[par], sH);
    if (err != cudaSuccess) return cuda_fail(err, "ensemble droplet-side launch");
    err = cudaStreamWaitEvent(sL, evNear[par ^ 1], 0);
    if (err == cudaSuccess && recentre) err = cudaStreamWaitEvent(sL, evCentre, 0);
    if (err == cudaSuccess) err = iblb::launch_ensemble_far(e->v, step, sL);
    if (err == cudaSuccess) err = cudaEventRecord(evFar[par], sL);
    if (err != cudaSuccess) return cuda_fail(err, "ensemble lattice launch");
    err = iblb::launch_ensemble_interp(e->v, sH, e->hi_prio);
    if (err != cudaSuccess) return cuda_fail(err, "ensemble interpolation launch");
    bool reg = false, obs = false;
    for (ibl_lb *lb : e->m) {
        ibl_mesh *mm = lb->mesh;
        if (mm->reg_every > 0 && next % mm->reg_every == 0) {
            // rewrites the member's patch of the next step: the next outside update waits for it
            err = iblb::launch_regularize(lb->v, mm->v, mm->reg, (int)(next % 3), sH, e->hi_prio);
            if (err != cudaSuccess) return cuda_fail(err, "ensemble regularisation launch");
            reg = true;
        }
    }
    if (reg) {
        err = cudaEventRecord(evNear[par], sH);
        if (err != cudaSuccess) return cuda_fail(err, "ensemble event");
    }
    std::vector<char> due(e->m.size(), 0);
    for (size_t k = 0; k < e->m.size(); ++k) {
        const ibl_mesh *mm = e->m[k]->mesh;
        due[k] = mm->readout_every > 0 && next % mm->readout_every == 0;
        obs = obs || due[k];
    }
    if (obs) {
        // the records read each member's step counter, closed by the outside update
        err = cudaStreamWaitEvent(sH, evFar[par], 0);
        if (err == cudaSuccess) err = iblb::launch_observables_batched(e->v, due, sH, e->hi_prio);
        if (err == cudaSuccess) err = cudaEventRecord(evNear[par], sH);
        if (err != cudaSuccess) return cuda_fail(err, "ensemble observables launch");
    }
    for (ibl_lb *lb : e->m) lb->host_step = next;
    return IBL_OK;
}

// Captures n ensemble steps (from the members' current step) into *out.
int ensemble_capture(ibl_ensemble *e, int n, cudaGraphExec_t *out)
{
    int st = ensemble_streams(e);
    if (st != IBL_OK) return st;
    std::vector<long long> saved;
    for (ibl_lb *lb : e->m) saved.push_back(lb->host_step);
    cudaStream_t cL = e->cap_stream, cH = e->cap_helper;
    cudaError_t err = cudaStreamBeginCapture(cL, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return cuda_fail(err, "begin capture");
    e->capturing = true;
    err = join(cL, cH, e->cFork);
    for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
        err = cudaEventRecord(e->cNear[k], cH);
        if (err == cudaSuccess) err = cudaEventRecord(e->cFar[k], cL);
    }
    if (err != cudaSuccess) st = cuda_fail(err, "capture fork");
    for (int k = 0; k < n && st == IBL_OK; ++k) st = ensemble_one_step(e, cL, cH);
    if (st == IBL_OK) {
        err = join(cH, cL, e->cJoin);
        if (err != cudaSuccess) st = cuda_fail(err, "capture join");
    }
    e->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cL, &g);
    if (e2 != cudaSuccess && st == IBL_OK) st = cuda_fail(e2, "end capture");
    if (st == IBL_OK) {
        const cudaError_t e3 = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
        if (e3 != cudaSuccess) st = cuda_fail(e3, "graph instantiate");
    }
    if (g) cudaGraphDestroy(g);
    for (size_t k = 0; k < e->m.size(); ++k) e->m[k]->host_step = saved[k];
    return st;
}

void ensemble_drop_graphs(ibl_ensemble *e)
{
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    e->gexec = nullptr;
    e->chunk = 0;
}


// ---- discrete adjoint: workspace layout and checkpoints --------------------
// A checkpoint holds what the next steps read of the state: the populations
// (in their AA slot layout), the control block (step, frame, patches), the
// node positions and the bounding-box rows the next force kernel reduces.
// The force field is zero between steps and the velocity field is written
// before it is read, so neither is saved.
struct AdjLayout {
    size_t lam[2] = {0, 0}, lam_u = 0, lam_F = 0, rec = 0, traj = 0, lam_r = 0, a_part = 0, s_part = 0, acc = 0,
           obs = 0, t0 = 0, ck = 0, total = 0;
    int lat_blocks = 0, near_blocks = 0, tri_blocks = 0;
    size_t rec_step = 0, traj_step = 0;                  // bytes per recorded step
    size_t traj_ctl = 0;                                 // control block copy inside a trajectory slot
    size_t ck_f = 0, ck_ctl = 0, ck_r = 0, ck_part = 0;  // offsets inside one checkpoint
    size_t f_bytes = 0, r_bytes = 0, part_bytes = 0, ck_step = 0;
    long long n_seg = 0;
    long long kmax = 0;                                  // steps per slot set
};

bool adj_layout(const ibl_lb *lb, const ibl_mesh *m, long long T, int K, AdjLayout &A)
{
    if (!lb || !m || T < 1 || K < 1) return false;
    const size_t es = lb->p.precision == IBL_FP64 ? 8 : 4;
    const size_t nodes = (size_t)lb->v.nodes;
    const int nv = m->v.nv, nt = m->v.nt;
    A.n_seg = (T + K - 1) / K;
    const long long kmax = std::min<long long>(K, T);
    A.f_bytes = es * 19 * (size_t)lb->v.qs;
    A.r_bytes = sizeof(double) * 3 * (size_t)nv;
    A.part_bytes = m->lay.obs_part - m->lay.part;
    A.ck_f = 0;
    A.ck_ctl = align256(A.f_bytes);
    A.ck_r = A.ck_ctl + align256(sizeof(Ctl));
    A.ck_part = A.ck_r + align256(A.r_bytes);
    A.ck_step = A.ck_part + align256(A.part_bytes);
    A.rec_step = align256(es * 7 * nodes);
    A.traj_ctl = align256(A.r_bytes);
    A.traj_step = A.traj_ctl + align256(sizeof(Ctl));
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = align256(off + b);
        return o;
    };
    A.lam[0] = take(es * 19 * nodes);
    A.lam[1] = take(es * 19 * nodes);
    A.lam_u = take(es * 4 * nodes);  // [nodes][4] records, as the forward force and velocity
    A.lam_F = take(es * 4 * nodes);
    A.lam_r = take(A.r_bytes);
    iblb::adj_grid(lb->v, nt, &A.lat_blocks, &A.near_blocks, &A.tri_blocks);
    A.a_part = take(sizeof(double) * 9 * (size_t)lb->v.n_frames * (size_t)(A.lat_blocks + A.near_blocks));
    A.s_part = take(sizeof(double) * (size_t)A.tri_blocks);
    A.acc = take(sizeof(double) * (1 + 9 * (size_t)lb->v.n_frames));
    A.obs = take(sizeof(double) * 11);
    A.t0 = take(sizeof(long long));
    // two slot sets: one segment is recorded while the next is swept back
    A.kmax = kmax;
    A.rec = take(A.rec_step * (size_t)kmax * 2);
    A.traj = take(A.traj_step * (size_t)kmax * 2);
    A.ck = take(A.ck_step * (size_t)(A.n_seg + 1));
    A.total = off;
    return true;
}

cudaError_t adj_save(ibl_lb *lb, const AdjLayout &A, char *ws, long long k, cudaStream_t s)
{
    char *c = ws + A.ck + A.ck_step * (size_t)k;
    const ibl_mesh *m = lb->mesh;
    cudaError_t e = cudaMemcpyAsync(c + A.ck_f, lb->v.f, A.f_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c + A.ck_ctl, lb->v.ctl, sizeof(Ctl), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c + A.ck_r, m->v.r, A.r_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c + A.ck_part, m->v.part, A.part_bytes, cudaMemcpyDeviceToDevice, s);
    return e;
}

cudaError_t adj_restore(ibl_lb *lb, const AdjLayout &A, const char *ws, long long k, cudaStream_t s)
{
    const char *c = ws + A.ck + A.ck_step * (size_t)k;
    const ibl_mesh *m = lb->mesh;
    cudaError_t e = cudaMemcpyAsync(lb->v.f, c + A.ck_f, A.f_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lb->v.ctl, c + A.ck_ctl, sizeof(Ctl), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->v.r, c + A.ck_r, A.r_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->v.part, c + A.ck_part, A.part_bytes, cudaMemcpyDeviceToDevice, s);
    return e;
}

}  // namespace

extern "C" {

const char *ibl_last_error(void) { return g_err.c_str(); }

int ibl_patch(ibl_lb *lb, int32_t lo[3], int32_t ext[3])
{
    if (!lb || !lo || !ext) return fail(IBL_EINVAL, "null argument");
    Ctl c;
    cudaError_t e = cudaMemcpyAsync(&c, lb->v.ctl, sizeof c, cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "patch readout");
    const int b = (int)(lb->host_step % 3);
    for (int a = 0; a < 3; ++a) {
        lo[a] = c.patch_lo[b][a];
        ext[a] = c.patch_ext[b][a];
    }
    return IBL_OK;
}

int ibl_velocity_set(int32_t *c, double *w)
{
    int cc[19][3];
    double ww[19];
    iblb::velocity_table(cc, ww);
    for (int i = 0; i < 19; ++i) {
        if (c)
            for (int a = 0; a < 3; ++a) c[3 * i + a] = cc[i][a];
        if (w) w[i] = ww[i];
    }
    return IBL_OK;
}

int ibl_lb_workspace_size(const ibl_lb_params *p, int n_frames, size_t *bytes)
{
    Layout L;
    if (!bytes) return fail(IBL_EINVAL, "null argument");
    if (!lb_layout(p, n_frames, L)) return fail(IBL_EINVAL, "invalid lattice parameters");
    *bytes = L.total;
    return IBL_OK;
}

int ibl_lb_create(const ibl_lb_params *p, const double *A_frames, int n_frames, int steps_per_frame, void *workspace,
                  size_t bytes, void *stream, ibl_lb **out)
{
    Layout L;
    if (!out || !A_frames) return fail(IBL_EINVAL, "null argument");
    if (!lb_layout(p, n_frames, L)) return fail(IBL_EINVAL, "invalid lattice parameters (version, sizes, bc, precision)");
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(IBL_EINVAL, "tau must be > 1/2");
    if (p->edge_rule != IBL_EDGE_COUNTER_SLIP && p->edge_rule != IBL_EDGE_PAPER_LITERAL)
        return fail(IBL_EINVAL, "unknown edge rule");
    if (steps_per_frame < 1) return fail(IBL_EINVAL, "steps_per_frame must be >= 1");
    for (int k = 0; k < 9 * n_frames; ++k)
        if (!std::isfinite(A_frames[k])) return fail(IBL_EINVAL, "non-finite velocity gradient");
    if (!workspace || bytes < L.total) return fail(IBL_ENOMEM, "lattice workspace too small");
    if (((uintptr_t)workspace & 255) != 0) return fail(IBL_EINVAL, "workspace must be 256-byte aligned");
    ibl_lb *lb = new ibl_lb();
    lb->p = *p;
    lb->lay = L;
    lb->ws = static_cast<char *>(workspace);
    lb->stream = static_cast<cudaStream_t>(stream);
    const long long nodes = (long long)p->n[0] * p->n[1] * p->n[2];
    LbView &v = lb->v;
    for (int a = 0; a < 3; ++a) {
        v.n[a] = p->n[a];
        v.bc[a] = p->bc[a];
    }
    v.nodes = (int)nodes;
    v.qs = pop_stride(nodes);
    v.precision = p->precision;
    v.rule = p->edge_rule;
    v.omega = 1.0 / p->tau;
    v.omega_f = (float)(1.0 / p->tau);
    v.inv_nx = 1.0f / (float)p->n[0];
    v.f = lb->ws + L.f;
    v.force = lb->ws + L.force;
    v.vel = lb->ws + L.vel;
    v.rec = p->record_fields ? lb->ws + L.rec : nullptr;
    v.visc = 0;
    v.omega_in = v.omega;
    v.omega_in_f = v.omega_f;
    v.ind = reinterpret_cast<unsigned int *>(lb->ws + L.ind);
    v.frames = reinterpret_cast<const double *>(lb->ws + L.frames);
    v.frames_t = lb->ws + L.frames_t;
    v.n_frames = n_frames;
    v.n_hold = steps_per_frame;
    v.ctl = reinterpret_cast<Ctl *>(lb->ws + L.ctl);
    v.staged = 0;
    v.stage_fault = 0;
    v.prefetch = 1;
    Ctl c;
    std::memset(&c, 0, sizeof c);
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 4; ++a) {
            c.patch_lo[b][a] = 0;
            c.patch_ext[b][a] = -1;
        }
    const size_t es = p->precision == IBL_FP64 ? 8 : 4;
    cudaError_t e = cudaMemcpyAsync(v.ctl, &c, sizeof c, cudaMemcpyHostToDevice, lb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lb->ws + L.frames, A_frames, sizeof(double) * 9 * n_frames, cudaMemcpyHostToDevice,
                            lb->stream);
    if (e == cudaSuccess) e = iblb::launch_convert_frames(v, 0, n_frames, lb->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.force, 0, es * 4 * nodes, lb->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.vel, 0, es * 4 * nodes, lb->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.ind, 0, ((size_t)nodes + 3) / 4 * 4, lb->stream);
    if (e == cudaSuccess && v.rec) e = cudaMemsetAsync(v.rec, 0, es * 7 * nodes, lb->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.f, 0, es * 19 * v.qs, lb->stream);
    if (e == cudaSuccess) e = iblb::launch_init(v, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);  // the host control block is a temporary
    if (e != cudaSuccess) {
        delete lb;
        return cuda_fail(e, "lattice initialisation");
    }
    *out = lb;
    return IBL_OK;
}

void ibl_lb_destroy(ibl_lb *lb)
{
    if (!lb) return;
    cudaStreamSynchronize(lb->stream);
    if (lb->mesh) lb->mesh->lb = nullptr;
    delete lb;
}

int ibl_set_frame(ibl_lb *lb, int k, const double *A)
{
    if (!lb || !A) return fail(IBL_EINVAL, "null argument");
    if (k < 0 || k >= lb->v.n_frames) return fail(IBL_EINVAL, "frame index out of range");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(A[i])) return fail(IBL_EINVAL, "non-finite velocity gradient");
    cudaError_t e = cudaMemcpyAsync(lb->ws + lb->lay.frames + sizeof(double) * 9 * (size_t)k, A, sizeof(double) * 9,
                                    cudaMemcpyHostToDevice, lb->stream);
    if (e == cudaSuccess) e = iblb::launch_convert_frames(lb->v, k, k + 1, lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "frame upload");
    return IBL_OK;
}

int ibl_icosphere_size(int level, int *n_nodes, int *n_tris)
{
    if (level < 0 || level > 9) return fail(IBL_EINVAL, "icosphere level must be in 0..9");
    long long p = 1;
    for (int l = 0; l < level; ++l) p *= 4;
    if (n_nodes) *n_nodes = (int)(10 * p + 2);
    if (n_tris) *n_tris = (int)(20 * p);
    return IBL_OK;
}

int ibl_icosphere(int level, double R, const double *center, double *r, int32_t *tris)
{
    if (level < 0 || level > 7 || !center || !r || !tris) return fail(IBL_EINVAL, "bad icosphere request");
    std::vector<double> xyz;
    std::vector<int> tri;
    icosphere(level, xyz, tri);
    for (size_t i = 0; i < xyz.size() / 3; ++i)
        for (int a = 0; a < 3; ++a) r[3 * i + a] = xyz[3 * i + a] * R + center[a];
    for (size_t k = 0; k < tri.size(); ++k) tris[k] = tri[k];
    return IBL_OK;
}

int ibl_mesh_workspace_size(int n_nodes, int n_tris, size_t *bytes)
{
    MeshLayout L;
    if (!bytes) return fail(IBL_EINVAL, "null argument");
    if (!mesh_layout(n_nodes, n_tris, L)) return fail(IBL_EINVAL, "bad mesh size");
    *bytes = L.total;
    return IBL_OK;
}

int ibl_mesh_create_icosphere(ibl_lb *lb, int level, double R, double sigma, const double *center, void *workspace,
                              size_t bytes, ibl_mesh **out)
{
    if (!lb) return fail(IBL_EINVAL, "null lattice");
    if (level < 0 || level > 7) return fail(IBL_EINVAL, "icosphere level must be in 0..7");
    if (!(R > 0) || !std::isfinite(R)) return fail(IBL_EINVAL, "radius must be > 0");
    std::vector<double> xyz;
    std::vector<int> tri;
    icosphere(level, xyz, tri);
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = center ? center[a] : 0.5 * (lb->p.n[a] - 1);
    for (size_t i = 0; i < xyz.size() / 3; ++i)
        for (int a = 0; a < 3; ++a) xyz[3 * i + a] = xyz[3 * i + a] * R + c[a];
    return mesh_attach(lb, (int)(xyz.size() / 3), xyz.data(), (int)(tri.size() / 3), tri.data(), sigma, workspace,
                       bytes, out);
}

int ibl_mesh_create(ibl_lb *lb, int n_nodes, const double *r, int n_tris, const int32_t *tris, double sigma,
                    void *workspace, size_t bytes, ibl_mesh **out)
{
    return mesh_attach(lb, n_nodes, r, n_tris, reinterpret_cast<const int *>(tris), sigma, workspace, bytes, out);
}

void ibl_mesh_destroy(ibl_mesh *m)
{
    if (!m) return;
    if (m->lb) {
        cudaStreamSynchronize(m->lb->stream);
        drop_graph(m->lb);
        m->lb->mesh = nullptr;
        m->lb->v.recentre = 0;  // the centre came from this droplet
        m->lb->v.visc = 0;      // and the inside flags
        m->lb->v.prefetch = 1;
    }
    delete m;
}

int ibl_set_viscosity_ratio(ibl_mesh *m, double chi)
{
    if (!m || !m->lb) return fail(IBL_EINVAL, "the mesh is not attached to a lattice");
    if (!(chi > 0.0) || !std::isfinite(chi)) return fail(IBL_EINVAL, "chi must be finite and > 0");
    ibl_lb *lb = m->lb;
    for (int a = 0; a < 3; ++a)
        if (lb->v.bc[a] != IBL_BC_ZOU_HE) return fail(IBL_EINVAL, "a viscosity ratio needs Zou-He walls on every axis");
    cudaStreamSynchronize(lb->stream);
    const double tau = 1.0 / lb->v.omega, tau_in = 0.5 + chi * (tau - 0.5);
    lb->v.visc = chi != 1.0 ? 1 : 0;
    lb->v.omega_in = 1.0 / tau_in;
    lb->v.omega_in_f = (float)(1.0 / tau_in);
    drop_graph(lb);  // captured chunks hold the lattice view by value
    return IBL_OK;
}

int ibl_set_recentring(ibl_mesh *m, int on)
{
    if (!m || !m->lb) return fail(IBL_EINVAL, "the mesh is not attached to a lattice");
    cudaStreamSynchronize(m->lb->stream);
    m->lb->v.recentre = on ? 1 : 0;
    drop_graph(m->lb);  // captured chunks hold the lattice view by value, and the step's dependencies change
    return IBL_OK;
}

int ibl_set_regularization(ibl_mesh *m, double alpha, double gamma, double tol, int max_iter, int every, int plus_sign)
{
    if (!m) return fail(IBL_EINVAL, "null mesh");
    if (!(alpha >= 0 && alpha <= 1) || !(gamma >= 0 && gamma <= 1) || !(tol > 0) || max_iter < 1 || every < 0)
        return fail(IBL_EINVAL, "regularisation parameters out of range");
    m->reg = iblb::RegParams{alpha, gamma, tol, max_iter, plus_sign ? 1 : 0, m->reg.trigger, m->reg.keep_volume};
    m->reg_every = every;
    if (m->lb) {
        cudaStreamSynchronize(m->lb->stream);
        drop_graph(m->lb);
    }
    return IBL_OK;
}

int ibl_set_regularization_trigger(ibl_mesh *m, double max_edge_ratio)
{
    if (!m || !(max_edge_ratio >= 0.0) || !std::isfinite(max_edge_ratio))
        return fail(IBL_EINVAL, "the trigger must be a finite ratio >= 0 (0 = always regularise)");
    if (max_edge_ratio > 0.0 && max_edge_ratio < 1.0) return fail(IBL_EINVAL, "an edge ratio below 1 never occurs");
    m->reg.trigger = max_edge_ratio;
    if (m->lb) {
        cudaStreamSynchronize(m->lb->stream);
        drop_graph(m->lb);  // captured chunks hold the parameters by value
    }
    return IBL_OK;
}

int ibl_set_regularization_keep_volume(ibl_mesh *m, int keep)
{
    if (!m) return fail(IBL_EINVAL, "null mesh");
    m->reg.keep_volume = keep ? 1 : 0;
    if (m->lb) {
        cudaStreamSynchronize(m->lb->stream);
        drop_graph(m->lb);  // captured chunks hold the parameters by value
    }
    return IBL_OK;
}

int ibl_regularization_stats(ibl_mesh *m, int *count, double *mesh_quality)
{
    if (!m || !m->lb) return fail(IBL_EINVAL, "null mesh");
    Ctl c;
    cudaError_t e = cudaMemcpyAsync(&c, m->lb->v.ctl, sizeof c, cudaMemcpyDeviceToHost, m->lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "regularisation stats");
    if (count) *count = c.reg_count;
    if (mesh_quality) *mesh_quality = c.mesh_q;
    return IBL_OK;
}

int ibl_set_readout(ibl_mesh *m, int every)
{
    if (!m || every < 0) return fail(IBL_EINVAL, "bad readout interval");
    m->readout_every = every;
    if (m->lb) {
        cudaStreamSynchronize(m->lb->stream);
        drop_graph(m->lb);
    }
    return IBL_OK;
}

int ibl_step(ibl_lb *lb, long long n)
{
    TraceRange trace_("ibl_step");
    if (!lb || n < 0) return fail(IBL_EINVAL, "bad step request");
    if (n == 0) return IBL_OK;
    int st = ensure_streams(lb);
    if (st != IBL_OK) return st;
    cudaStream_t sL = lb->stream, sH = lb->helper;
    // the helper stream starts after everything already on the bound stream
    cudaError_t e = join(sL, sH, lb->evFork);
    if (e != cudaSuccess) return cuda_fail(e, "stream fork");
    bool forked = true;  // eager steps may use the helper stream
    const int chunk = lb->graphs ? chunk_length(lb) : 0;
    if (chunk > 0 && lb->chunk != chunk) drop_graph(lb);
    std::vector<Piece> plan;
    plan_steps(lb, n, plan);
    // whole chunks and captured segments replay as graphs, other steps run
    // eagerly (consecutive eager steps pipeline across steps on the two
    // streams, while a graph boundary drains them); a graph starts after
    // all eager work
    auto replay = [&](cudaGraphExec_t g, long long len) -> int {
        if (forked) {
            e = join(sH, sL, lb->evJoin);
            if (e != cudaSuccess) return cuda_fail(e, "stream join");
            forked = false;
        }
        e = cudaGraphLaunch(g, sL);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        lb->host_step += len;
        lb->steps_replayed += len;
        return IBL_OK;
    };
    for (const Piece &pc : plan) {
        if (pc.chunk) {
            if (!lb->gexec[pc.slot]) {
                st = capture_chunk(lb, chunk, pc.slot);
                if (st != IBL_OK) return st;
            }
            st = replay(lb->gexec[pc.slot], pc.len);
            if (st != IBL_OK) return st;
            continue;
        }
        if (lb->graphs && pc.len >= 2) {
            // a segment met for the second time is captured (stepping in
            // fixed increments then replays graphs throughout once every
            // phase has come round twice)
            ibl_lb::Segment *sg = find_segment(lb, pc.phase, pc.len);
            if (!sg && seen_before(lb, pc.phase, pc.len)) {
                st = capture_segment(lb, pc, &sg);
                if (st != IBL_OK) return st;
            }
            if (sg) {
                st = replay(sg->g, pc.len);
                if (st != IBL_OK) return st;
                continue;
            }
        }
        for (long long k = 0; k < pc.len; ++k) {
            if (!forked) {
                e = join(sL, sH, lb->evFork);
                if (e != cudaSuccess) return cuda_fail(e, "stream fork");
                forked = true;
            }
            st = one_step(lb, false, sL, sH);
            if (st != IBL_OK) return st;
            ++lb->steps_eager;
        }
    }
    // the bound stream resumes after all helper-stream work
    if (forked) {
        e = join(sH, sL, lb->evJoin);
        if (e != cudaSuccess) return cuda_fail(e, "stream join");
    }
    return IBL_OK;
}

int ibl_prepare_steps(ibl_lb *lb, long long n)
{
    TraceRange trace_("ibl_prepare_steps");
    if (!lb || n < 0) return fail(IBL_EINVAL, "bad step request");
    if (!lb->graphs || n == 0) return IBL_OK;
    const int chunk = chunk_length(lb);
    if (chunk > 0 && lb->chunk != chunk) drop_graph(lb);
    std::vector<Piece> plan;
    plan_steps(lb, n, plan);
    const long long saved = lb->host_step;
    int st = IBL_OK;
    for (const Piece &pc : plan) {
        if (pc.chunk && !lb->gexec[pc.slot]) {
            lb->host_step = pc.start;
            st = capture_chunk(lb, chunk, pc.slot);
            lb->host_step = saved;
            if (st == IBL_OK) {
                const cudaError_t e = cudaGraphUpload(lb->gexec[pc.slot], lb->stream);
                if (e != cudaSuccess) st = cuda_fail(e, "graph upload");
            }
        } else if (!pc.chunk && pc.len >= 2 && !find_segment(lb, pc.phase, pc.len)) {
            ibl_lb::Segment *sg = nullptr;
            st = capture_segment(lb, pc, &sg);
        }
        if (st != IBL_OK) return st;
    }
    return IBL_OK;
}

int ibl_set_outside_update(ibl_lb *lb, int kind)
{
    if (!lb) return fail(IBL_EINVAL, "null lattice");
    if (kind < 0 || kind > iblb::kStagedShapes) return fail(IBL_EINVAL, "outside-update kind out of range");
    if (kind > 0 && !iblb::staged_ok(lb->v))
        return fail(IBL_EINVAL, "the staged outside update needs FP32 populations and Zou-He walls on every axis");
    cudaStreamSynchronize(lb->stream);
    const cudaError_t e = iblb::staged_prepare(kind);
    if (e != cudaSuccess) return cuda_fail(e, "staged kernel attributes");
    drop_graph(lb);  // captured chunks hold the lattice view by value
    lb->v.staged = kind;
    return IBL_OK;
}

int ibl_test_stage_timeout(ibl_lb *lb, int on)
{
    if (!lb) return fail(IBL_EINVAL, "null lattice");
    cudaStreamSynchronize(lb->stream);
    drop_graph(lb);  // captured chunks hold the lattice view by value
    lb->v.stage_fault = on ? 1 : 0;
    return IBL_OK;
}

int ibl_outside_update(const ibl_lb *lb, int *kind)
{
    if (!lb || !kind) return fail(IBL_EINVAL, "null argument");
    *kind = lb->v.staged;
    return IBL_OK;
}

int ibl_step_paths(const ibl_lb *lb, long long *eager, long long *replayed)
{
    if (!lb || !eager || !replayed) return fail(IBL_EINVAL, "null argument");
    *eager = lb->steps_eager;
    *replayed = lb->steps_replayed;
    return IBL_OK;
}

int ibl_set_graphs(ibl_lb *lb, int enable)
{
    if (!lb) return fail(IBL_EINVAL, "null lattice");
    cudaStreamSynchronize(lb->stream);
    drop_graph(lb);
    lb->graphs = enable != 0;
    return IBL_OK;
}

int ibl_step_record(ibl_lb *lb)
{
    TraceRange trace_("ibl_step_record");
    if (!lb) return fail(IBL_EINVAL, "null lattice");
    if (!lb->v.rec) return fail(IBL_EINVAL, "lattice created without record_fields");
    int st = ensure_streams(lb);
    if (st != IBL_OK) return st;
    cudaError_t e = join(lb->stream, lb->helper, lb->evFork);
    if (e != cudaSuccess) return cuda_fail(e, "stream fork");
    st = one_step(lb, true, lb->stream, lb->helper);
    if (st != IBL_OK) return st;
    e = join(lb->helper, lb->stream, lb->evJoin);
    if (e != cudaSuccess) return cuda_fail(e, "stream join");
    lb->recorded = true;
    return IBL_OK;
}

int ibl_sync(ibl_lb *lb)
{
    if (!lb) return fail(IBL_EINVAL, "null lattice");
    return lb_status_from_device(lb);
}

long long ibl_steps_done(const ibl_lb *lb) { return lb ? lb->host_step : -1; }

namespace {

// Checkpoint file: this header, the lattice workspace, then the mesh
// workspace.  Between steps the workspaces hold the whole dynamic state (the
// populations, the control block with its step counter, frame slots, patch
// buffers and error bits, the frames, the mesh positions, forces, bounding-box
// rows and shape-record ring); the Eulerian force, the velocity scratch and
// the inside flags are zero or unused there.
struct CkptHeader {
    char magic[8];
    int abi_version;
    int n[3], bc[3];
    int precision, edge_rule, record_fields;
    int n_frames, steps_per_frame;
    int mesh_nv, mesh_nt;  // -1 without a mesh
    double tau;
    long long host_step;
    unsigned long long lb_bytes, mesh_bytes;
};
const char kCkptMagic[8] = {'I', 'B', 'L', 'B', 'C', 'K', 'P', '1'};

CkptHeader ckpt_header(const ibl_lb *lb)
{
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kCkptMagic, sizeof h.magic);
    h.abi_version = IBL_ABI_VERSION;
    for (int a = 0; a < 3; ++a) {
        h.n[a] = lb->v.n[a];
        h.bc[a] = lb->v.bc[a];
    }
    h.precision = lb->p.precision;
    h.edge_rule = lb->p.edge_rule;
    h.record_fields = lb->p.record_fields ? 1 : 0;
    h.n_frames = lb->v.n_frames;
    h.steps_per_frame = lb->v.n_hold;
    h.mesh_nv = lb->mesh ? lb->mesh->v.nv : -1;
    h.mesh_nt = lb->mesh ? lb->mesh->v.nt : -1;
    h.tau = lb->p.tau;
    h.host_step = lb->host_step;
    h.lb_bytes = lb->lay.total;
    h.mesh_bytes = lb->mesh ? lb->mesh->lay.total : 0;
    return h;
}

char *mesh_ws(const ibl_mesh *m) { return reinterpret_cast<char *>(m->v.r) - m->lay.r; }

}  // namespace

int ibl_save(ibl_lb *lb, const char *path)
{
    if (!lb || !path) return fail(IBL_EINVAL, "null argument");
    cudaError_t e = cudaStreamSynchronize(lb->stream);
    if (e == cudaSuccess && lb->helper) e = cudaStreamSynchronize(lb->helper);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    const CkptHeader h = ckpt_header(lb);
    std::vector<char> buf(h.lb_bytes + h.mesh_bytes);
    e = cudaMemcpy(buf.data(), lb->ws, h.lb_bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && lb->mesh)
        e = cudaMemcpy(buf.data() + h.lb_bytes, mesh_ws(lb->mesh), h.mesh_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
    std::FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(IBL_EINVAL, std::string("cannot open for writing: ") + path);
    const bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1 && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    const bool closed = std::fclose(fp) == 0;
    if (!ok || !closed) return fail(IBL_EINVAL, std::string("cannot write: ") + path);
    return IBL_OK;
}

int ibl_load(ibl_lb *lb, const char *path)
{
    if (!lb || !path) return fail(IBL_EINVAL, "null argument");
    std::FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(IBL_EINVAL, std::string("cannot open: ") + path);
    CkptHeader h;
    if (std::fread(&h, sizeof h, 1, fp) != 1) {
        std::fclose(fp);
        return fail(IBL_EINVAL, "not a checkpoint (short header)");
    }
    const CkptHeader mine = ckpt_header(lb);
    const bool same = std::memcmp(h.magic, kCkptMagic, sizeof h.magic) == 0 && h.abi_version == mine.abi_version &&
                      std::memcmp(h.n, mine.n, sizeof h.n) == 0 && std::memcmp(h.bc, mine.bc, sizeof h.bc) == 0 &&
                      h.precision == mine.precision && h.edge_rule == mine.edge_rule &&
                      h.record_fields == mine.record_fields && h.n_frames == mine.n_frames &&
                      h.steps_per_frame == mine.steps_per_frame && h.mesh_nv == mine.mesh_nv &&
                      h.mesh_nt == mine.mesh_nt && h.tau == mine.tau && h.lb_bytes == mine.lb_bytes &&
                      h.mesh_bytes == mine.mesh_bytes && h.host_step >= 0;
    if (!same) {
        std::fclose(fp);
        return fail(IBL_EINVAL, "checkpoint does not match this lattice and mesh (box, boundaries, precision, "
                                "edge rule, tau, frames or mesh size)");
    }
    std::vector<char> buf(h.lb_bytes + h.mesh_bytes);
    const bool ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    std::fclose(fp);
    if (!ok) return fail(IBL_EINVAL, "truncated checkpoint");
    cudaError_t e = cudaStreamSynchronize(lb->stream);
    if (e == cudaSuccess && lb->helper) e = cudaStreamSynchronize(lb->helper);
    if (e == cudaSuccess) e = cudaMemcpy(lb->ws, buf.data(), h.lb_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && lb->mesh)
        e = cudaMemcpy(mesh_ws(lb->mesh), buf.data() + h.lb_bytes, h.mesh_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint upload");
    lb->host_step = h.host_step;
    drop_graph(lb);  // chunks are captured for a phase of the step sequence
    return IBL_OK;
}

int ibl_readout(ibl_mesh *m, ibl_observables *out)
{
    TraceRange trace_("ibl_readout");
    if (!m || !m->lb || !out) return fail(IBL_EINVAL, "null argument");
    ibl_lb *lb = m->lb;
    cudaError_t e = iblb::launch_observables(lb->v, m->v, lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "observables launch");
    Ctl c;
    e = cudaMemcpyAsync(&c, lb->v.ctl, sizeof c, cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "observables readout");
    const int slot = (c.n_records - 1) % m->v.ring_cap;
    e = cudaMemcpyAsync(out, m->v.ring + slot, sizeof(ibl_observables), cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "observables copy");
    return lb_status_from_device(lb);
}

int ibl_read_series(ibl_mesh *m, ibl_observables *out, int max, int *count)
{
    if (!m || !m->lb || !out || !count || max < 0) return fail(IBL_EINVAL, "null argument");
    ibl_lb *lb = m->lb;
    Ctl c;
    cudaError_t e = cudaMemcpyAsync(&c, lb->v.ctl, sizeof c, cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "series readout");
    const int cap = m->v.ring_cap;
    const int have = std::min(c.n_records, cap);
    const int first = c.n_records - have;
    std::vector<ibl_observables> ring(cap);
    e = cudaMemcpyAsync(ring.data(), m->v.ring, sizeof(ibl_observables) * cap, cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "series copy");
    const int n = std::min(have, max);
    for (int k = 0; k < n; ++k) out[k] = ring[(first + k) % cap];
    *count = n;
    return lb_status_from_device(lb);
}

int ibl_copy_fields(ibl_lb *lb, double *rho, double *u, double *F)
{
    if (!lb) return fail(IBL_EINVAL, "null lattice");
    if (!lb->v.rec || !lb->recorded) return fail(IBL_EINVAL, "no recorded step (use ibl_step_record)");
    const size_t nodes = (size_t)lb->v.nodes;
    const bool dbl = lb->p.precision == IBL_FP64;
    const size_t es = dbl ? 8 : 4;
    std::vector<char> h(es * 7 * nodes);
    cudaError_t e = cudaMemcpyAsync(h.data(), lb->v.rec, h.size(), cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "field copy");
    auto at = [&](size_t k) -> double {
        return dbl ? reinterpret_cast<const double *>(h.data())[k] : (double)reinterpret_cast<const float *>(h.data())[k];
    };
    for (size_t i = 0; i < nodes; ++i) {
        if (rho) rho[i] = 1.0 + at(i);
        for (int a = 0; a < 3; ++a) {
            if (u) u[a * nodes + i] = at((1 + a) * nodes + i);
            if (F) F[a * nodes + i] = at((4 + a) * nodes + i);
        }
    }
    return lb_status_from_device(lb);
}

int ibl_copy_populations(ibl_lb *lb, double *f)
{
    if (!lb || !f) return fail(IBL_EINVAL, "null argument");
    const int nx = lb->p.n[0], ny = lb->p.n[1], nz = lb->p.n[2];
    const size_t nodes = (size_t)lb->v.nodes, qs = (size_t)lb->v.qs;
    const bool dbl = lb->p.precision == IBL_FP64;
    const size_t es = dbl ? 8 : 4;
    std::vector<char> h(es * 19 * qs);
    cudaError_t e = cudaMemcpyAsync(h.data(), lb->v.f, h.size(), cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "population copy");
    auto at = [&](size_t k) -> double {
        return dbl ? reinterpret_cast<const double *>(h.data())[k] : (double)reinterpret_cast<const float *>(h.data())[k];
    };
    int c[19][3];
    double w[19];
    iblb::velocity_table(c, w);
    const bool swapped = (lb->host_step & 1) != 0;
    const int nn[3] = {nx, ny, nz};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t id = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
                const int xyz[3] = {x, y, z};
                for (int i = 0; i < 19; ++i) {
                    int s[3];
                    bool inside = true;
                    for (int a = 0; a < 3; ++a) {
                        s[a] = xyz[a] - c[i][a];
                        if (lb->p.bc[a] == IBL_BC_PERIODIC) s[a] = (s[a] + nn[a]) % nn[a];
                        else if (s[a] < 0 || s[a] >= nn[a]) inside = false;
                    }
                    double v = 0.0;
                    if (inside) {
                        if (!swapped) {
                            v = w[i] + at((size_t)i * qs + id);
                        } else {
                            const int o = i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9);
                            const size_t sid = (size_t)s[0] + (size_t)nx * ((size_t)s[1] + (size_t)ny * s[2]);
                            v = w[i] + at((size_t)o * qs + sid);
                        }
                    }
                    f[(size_t)i * nodes + id] = v;
                }
            }
    return IBL_OK;
}

int ibl_copy_mesh(ibl_mesh *m, double *r, double *F, int32_t *tris)
{
    if (!m || !m->lb) return fail(IBL_EINVAL, "null mesh");
    cudaStream_t s = m->lb->stream;
    cudaError_t e = cudaSuccess;
    if (r) e = cudaMemcpyAsync(r, m->v.r, sizeof(double) * 3 * m->v.nv, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && F) e = cudaMemcpyAsync(F, m->v.fn, sizeof(double) * 3 * m->v.nv, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mesh copy");
    if (tris) std::memcpy(tris, m->tris.data(), sizeof(int) * m->tris.size());
    return IBL_OK;
}

int ibl_copy_neighbours(ibl_mesh *m, int32_t *ptr, int32_t *idx, int *nnz)
{
    if (!m) return fail(IBL_EINVAL, "null mesh");
    if (ptr) std::memcpy(ptr, m->nb_ptr.data(), sizeof(int) * m->nb_ptr.size());
    if (idx) std::memcpy(idx, m->nb_idx.data(), sizeof(int) * m->nb_idx.size());
    if (nnz) *nnz = (int)m->nb_idx.size();
    return IBL_OK;
}

int ibl_regularize_now(ibl_mesh *m, int *iters)
{
    TraceRange trace_("ibl_regularize_now");
    if (!m || !m->lb) return fail(IBL_EINVAL, "null mesh");
    ibl_lb *lb = m->lb;
    iblb::RegParams now = m->reg;
    now.trigger = 0.0;  // unconditional, whatever the schedule's trigger
    cudaError_t e = iblb::launch_regularize(lb->v, m->v, now, (int)(lb->host_step % 3), lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "regularisation launch");
    Ctl c;
    e = cudaMemcpyAsync(&c, lb->v.ctl, sizeof c, cudaMemcpyDeviceToHost, lb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "regularisation readout");
    if (iters) *iters = c.reg_iters;
    return lb_status_from_device(lb);
}

int ibl_run_frames(ibl_lb *lb, ibl_mesh *m, const double *A_frames, int n_frames, int steps_per_frame,
                   ibl_observables *out)
{
    TraceRange trace_("ibl_run_frames");
    if (!lb || !m || m->lb != lb || !A_frames || !out || n_frames < 0) return fail(IBL_EINVAL, "bad arguments");
    if (steps_per_frame != lb->v.n_hold) return fail(IBL_EINVAL, "steps_per_frame differs from the lattice's");
    if (lb->host_step % lb->v.n_hold != 0) return fail(IBL_EINVAL, "step count is not at a frame boundary");
    for (int k = 0; k < n_frames; ++k) {
        const long long fk = lb->host_step / lb->v.n_hold;
        if (fk >= lb->v.n_frames) return fail(IBL_EINVAL, "frame capacity of the lattice exceeded");
        int st = ibl_set_frame(lb, (int)fk, A_frames + 9 * (size_t)k);
        if (st != IBL_OK) return st;
        st = ibl_step(lb, steps_per_frame);
        if (st != IBL_OK) return st;
        cudaError_t e = iblb::launch_observables(lb->v, m->v, lb->stream);
        if (e != cudaSuccess) return cuda_fail(e, "observables launch");
        Ctl c;
        e = cudaMemcpyAsync(&c, lb->v.ctl, sizeof c, cudaMemcpyDeviceToHost, lb->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
        if (e != cudaSuccess) return cuda_fail(e, "frame readout");
        const int slot = (c.n_records - 1) % m->v.ring_cap;
        e = cudaMemcpyAsync(out + k, m->v.ring + slot, sizeof(ibl_observables), cudaMemcpyDeviceToHost, lb->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lb->stream);
        if (e != cudaSuccess) return cuda_fail(e, "frame record copy");
        if (c.err) return lb_status_from_device(lb);
    }
    return IBL_OK;
}

int ibl_ensemble_workspace_size(int n, ibl_lb *const *members, size_t *bytes)
{
    if (!bytes) return fail(IBL_EINVAL, "null argument");
    EnsembleLayout L;
    std::string why;
    const int st = ensemble_layout(n, members, L, why);
    if (st != IBL_OK) return fail(st, why);
    *bytes = L.total;
    return IBL_OK;
}

int ibl_ensemble_create(int n, ibl_lb *const *members, void *workspace, size_t bytes, ibl_ensemble **out)
{
    if (!out) return fail(IBL_EINVAL, "null argument");
    EnsembleLayout L;
    std::string why;
    const int st = ensemble_layout(n, members, L, why);
    if (st != IBL_OK) return fail(st, why);
    if (!workspace || bytes < L.total) return fail(IBL_ENOMEM, "ensemble workspace too small");
    if (((uintptr_t)workspace & 255) != 0) return fail(IBL_EINVAL, "workspace must be 256-byte aligned");
    const ibl_lb *m0 = members[0];
    std::vector<LbView> lv;
    std::vector<MeshView> mv;
    std::vector<int> lat_member[2], lat_start[2], node_member, node_start;
    for (int k = 0; k < n; ++k) {
        const ibl_lb *lb = members[k];
        if (lb->p.precision != m0->p.precision) return fail(IBL_EINVAL, "members differ in precision");
        if (lb->stream != m0->stream) return fail(IBL_EINVAL, "members are bound to different streams");
        if (lb->host_step != m0->host_step) return fail(IBL_EINVAL, "members are at different step counts");
        if (lb->v.visc) return fail(IBL_EINVAL, "ensemble members need chi = 1");
        for (int j = 0; j < k; ++j)
            if (members[j] == lb) return fail(IBL_EINVAL, "a lattice appears twice");
        lv.push_back(lb->v);
        mv.push_back(lb->mesh->v);
        for (int t = 0; t < 2; ++t) {
            lat_start[t].push_back((int)lat_member[t].size());
            for (long long b = 0; b < lattice_blocks(lb, t == 0 ? 128 : 256); ++b) lat_member[t].push_back(k);
        }
        node_start.push_back((int)node_member.size());
        for (int b = 0; b < (lb->mesh->v.nv + iblb::kFwdNodesPerBlock - 1) / iblb::kFwdNodesPerBlock; ++b)
            node_member.push_back(k);
    }
    for (int t = 0; t < 2; ++t) lat_start[t].push_back((int)lat_member[t].size());
    node_start.push_back((int)node_member.size());
    char *w = static_cast<char *>(workspace);
    cudaStream_t s = m0->stream;
    cudaError_t e = cudaSuccess;
    auto up = [&](size_t off, const void *src, size_t nbytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(w + off, src, nbytes, cudaMemcpyHostToDevice, s);
    };
    for (int t = 0; t < 2; ++t) {
        up(L.lat_member[t], lat_member[t].data(), sizeof(int) * lat_member[t].size());
        up(L.lat_start[t], lat_start[t].data(), sizeof(int) * lat_start[t].size());
    }
    up(L.node_member, node_member.data(), sizeof(int) * node_member.size());
    up(L.node_start, node_start.data(), sizeof(int) * node_start.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host tables are temporaries
    if (e != cudaSuccess) return cuda_fail(e, "ensemble upload");
    ibl_ensemble *en = new ibl_ensemble();
    en->m.assign(members, members + n);
    en->stream = s;
    iblb::EnsembleView &v = en->v;
    v.lv = lv;
    v.mv = mv;
    for (int t = 0; t < 2; ++t) {
        v.lat_member[t] = reinterpret_cast<const int *>(w + L.lat_member[t]);
        v.lat_start_d[t] = reinterpret_cast<const int *>(w + L.lat_start[t]);
        v.lat_start[t] = lat_start[t];
    }
    v.node_member = reinterpret_cast<const int *>(w + L.node_member);
    v.node_start_d = reinterpret_cast<const int *>(w + L.node_start);
    v.node_start = node_start;
    v.precision = m0->p.precision;
    v.shape = iblb::kEnsDefaultShape;
    *out = en;
    return IBL_OK;
}

int ibl_ensemble_step(ibl_ensemble *en, long long n)
{
    TraceRange trace_("ibl_ensemble_step");
    if (!en || n < 0) return fail(IBL_EINVAL, "bad ensemble step request");
    if (n == 0) return IBL_OK;
    const long long h0 = en->m[0]->host_step;
    for (ibl_lb *lb : en->m)
        if (lb->host_step != h0 || !lb->mesh) return fail(IBL_EINVAL, "members were stepped apart from the ensemble");
    int st = ensemble_streams(en);
    if (st != IBL_OK) return st;
    cudaStream_t sL = en->stream, sH = en->helper;
    cudaError_t e = join(sL, sH, en->evFork);
    if (e != cudaSuccess) return cuda_fail(e, "stream fork");
    bool forked = true;
    const int chunk = ensemble_chunk(en);
    long long done = 0;
    auto replay = [&](cudaGraphExec_t g, int len) -> int {
        if (forked) {
            e = join(sH, sL, en->evJoin);
            if (e != cudaSuccess) return cuda_fail(e, "stream join");
            forked = false;
        }
        e = cudaGraphLaunch(g, sL);
        if (e != cudaSuccess) return cuda_fail(e, "ensemble graph launch");
        for (ibl_lb *lb : en->m) lb->host_step += len;
        done += len;
        return IBL_OK;
    };
    while (done < n) {
        const long long s0 = en->m[0]->host_step;
        if (chunk > 0 && s0 % chunk == 0 && n - done >= chunk) {
            if (en->chunk != chunk || !en->gexec) {
                ensemble_drop_graphs(en);
                st = ensemble_capture(en, chunk, &en->gexec);
                if (st != IBL_OK) {
                    ensemble_drop_graphs(en);
                    return st;
                }
                en->chunk = chunk;
            }
            st = replay(en->gexec, chunk);
            if (st != IBL_OK) return st;
            continue;
        }
        if (!forked) {
            e = join(sL, sH, en->evFork);
            if (e != cudaSuccess) return cuda_fail(e, "stream fork");
            forked = true;
        }
        st = ensemble_one_step(en, sL, sH);
        if (st != IBL_OK) return st;
        ++done;
    }
    if (forked) {
        e = join(sH, sL, en->evJoin);
        if (e != cudaSuccess) return cuda_fail(e, "stream join");
    }
    return IBL_OK;
}

int ibl_ensemble_set_shape(ibl_ensemble *en, int shape)
{
    if (!en || shape < 0 || shape >= IBL_ENSEMBLE_SHAPES) return fail(IBL_EINVAL, "bad ensemble launch shape");
    cudaStreamSynchronize(en->stream);
    en->v.shape = shape;
    ensemble_drop_graphs(en);  // captured chunks hold the launch shape
    return IBL_OK;
}

int ibl_ensemble_shape(const ibl_ensemble *en, int *shape, int *threads, int *prefetch_waves)
{
    if (!en) return fail(IBL_EINVAL, "null ensemble");
    if (shape) *shape = en->v.shape;
    if (threads) *threads = iblb::ens_shape_threads(en->v.shape);
    if (prefetch_waves) *prefetch_waves = iblb::ens_shape_waves(en->v.shape);
    return IBL_OK;
}

int ibl_ensemble_tune(ibl_ensemble *en, int steps_per_candidate, double *ms, int *chosen)
{
    TraceRange trace_("ibl_ensemble_tune");
    if (!en || steps_per_candidate < 1) return fail(IBL_EINVAL, "bad tuning request");
    const long long h0 = en->m[0]->host_step;
    for (ibl_lb *lb : en->m)
        if (lb->host_step != h0 || !lb->mesh) return fail(IBL_EINVAL, "members were stepped apart from the ensemble");
    int st = ensemble_streams(en);
    if (st != IBL_OK) return st;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "tuning events");
    cudaStream_t sL = en->stream, sH = en->helper;
    double best = 1e300;
    int best_k = en->v.shape;
    for (int k = 0; k < IBL_ENSEMBLE_SHAPES && st == IBL_OK; ++k) {
        en->v.shape = k;
        float t = 0.f;
        for (int pass = 0; pass < 2 && st == IBL_OK; ++pass) {
            // pass 0: two untimed steps; pass 1: the timed ones
            const int n = pass == 0 ? 2 : steps_per_candidate;
            e = join(sL, sH, en->evFork);
            if (e == cudaSuccess && pass == 1) e = cudaEventRecord(a, sL);
            for (int j = 0; j < n && st == IBL_OK && e == cudaSuccess; ++j) st = ensemble_one_step(en, sL, sH);
            if (st == IBL_OK && e == cudaSuccess) e = join(sH, sL, en->evJoin);
            if (e == cudaSuccess && pass == 1) e = cudaEventRecord(b, sL);
            if (e == cudaSuccess) e = cudaStreamSynchronize(sL);
            if (e == cudaSuccess && pass == 1) e = cudaEventElapsedTime(&t, a, b);
            if (e != cudaSuccess) st = cuda_fail(e, "tuning run");
        }
        if (st != IBL_OK) break;
        const double per = (double)t / steps_per_candidate;
        if (ms) ms[k] = per;
        if (per < best) {
            best = per;
            best_k = k;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    en->v.shape = best_k;
    ensemble_drop_graphs(en);
    if (chosen) *chosen = best_k;
    if (st != IBL_OK) return st;
    return ibl_ensemble_sync(en);
}

int ibl_ensemble_sync(ibl_ensemble *en)
{
    if (!en) return fail(IBL_EINVAL, "null ensemble");
    for (size_t k = 0; k < en->m.size(); ++k) {
        const int st = lb_status_from_device(en->m[k]);
        if (st != IBL_OK) return fail(st, "ensemble member " + std::to_string(k) + ": " + g_err);
    }
    return IBL_OK;
}

void ibl_ensemble_destroy(ibl_ensemble *en)
{
    if (!en) return;
    cudaStreamSynchronize(en->stream);
    delete en;
}

int ibl_profile_enable(ibl_lb *lb, int mask, int every)
{
    if (!lb || mask < 0 || mask > 15 || every < 1) return fail(IBL_EINVAL, "bad profiling mask or stride");
    cudaStreamSynchronize(lb->stream);
    drop_graph(lb);  // a captured chunk may hold event nodes of the pool
    lb->prof.clear();
    lb->prof.mask = mask;
    lb->prof.every = every;
    return IBL_OK;
}

int ibl_profile_read(ibl_lb *lb, double ms[3], long long launches[3])
{
    if (!lb || !ms || !launches) return fail(IBL_EINVAL, "null argument");
    cudaError_t e = cudaStreamSynchronize(lb->stream);
    if (e != cudaSuccess) return cuda_fail(e, "profile synchronize");
    for (int k = 0; k < 3; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (auto &mk : lb->prof.marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, lb->prof.pool[mk.second], lb->prof.pool[mk.second + 1]) == cudaSuccess) {
            ms[mk.first] += t;
            launches[mk.first] += 1;
        }
    }
    return IBL_OK;
}

int ibl_adjoint_workspace_size(const ibl_lb *lb, long long n_steps, int K, size_t *bytes)
{
    AdjLayout A;
    if (!bytes) return fail(IBL_EINVAL, "null argument");
    if (!lb || !lb->mesh) return fail(IBL_EINVAL, "the lattice has no droplet");
    if (!adj_layout(lb, lb->mesh, n_steps, K, A)) return fail(IBL_EINVAL, "n_steps and K must be >= 1");
    *bytes = A.total;
    return IBL_OK;
}

int ibl_adjoint(ibl_lb *lb, long long n_steps, int K, void *workspace, size_t bytes, double *D, double *dD_dsigma,
                double *dD_dA, double *dD_dr0)
{
    TraceRange trace_("ibl_adjoint");
    if (!lb || !lb->mesh) return fail(IBL_EINVAL, "the lattice has no droplet");
    ibl_mesh *m = lb->mesh;
    AdjLayout A;
    if (!adj_layout(lb, m, n_steps, K, A)) return fail(IBL_EINVAL, "n_steps and K must be >= 1");
    if (lb->host_step != 0) return fail(IBL_EINVAL, "the adjoint starts from step 0");
    if (m->reg_every != 0) return fail(IBL_EINVAL, "the adjoint needs the regularisation switched off");
    if (lb->v.recentre) return fail(IBL_EINVAL, "the adjoint does not differentiate the re-centring");
    if (lb->v.visc) return fail(IBL_EINVAL, "the adjoint needs chi = 1");
    if (!workspace || bytes < A.total) return fail(IBL_ENOMEM, "adjoint workspace too small");
    if (((uintptr_t)workspace & 255) != 0) return fail(IBL_EINVAL, "workspace must be 256-byte aligned");
    int st = ensure_streams(lb);
    if (st != IBL_OK) return st;
    char *ws = static_cast<char *>(workspace);
    cudaStream_t s = lb->stream;
    const size_t es = lb->p.precision == IBL_FP64 ? 8 : 4;
    const size_t nodes = (size_t)lb->v.nodes;
    const int nf = lb->v.n_frames;
    iblb::AdjView J;
    J.lam_u = ws + A.lam_u;
    J.lam_F = ws + A.lam_F;
    J.lam_r = reinterpret_cast<double *>(ws + A.lam_r);
    J.a_part = reinterpret_cast<double *>(ws + A.a_part);
    J.s_part = reinterpret_cast<double *>(ws + A.s_part);
    J.lat_blocks = A.lat_blocks;
    J.acc_blocks = A.lat_blocks + A.near_blocks;
    J.tri_blocks = A.tri_blocks;
    J.acc = reinterpret_cast<double *>(ws + A.acc);
    J.obs = reinterpret_cast<double *>(ws + A.obs);
    J.t0 = reinterpret_cast<long long *>(ws + A.t0);
    void *lam[2] = {ws + A.lam[0], ws + A.lam[1]};
    cudaError_t e = cudaMemsetAsync(lam[0], 0, es * 19 * nodes, s);  // D does not depend on the final populations
    if (e == cudaSuccess) e = cudaMemsetAsync(J.lam_u, 0, es * 4 * nodes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(J.a_part, 0, sizeof(double) * 9 * (size_t)nf * J.acc_blocks, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(J.s_part, 0, sizeof(double) * (size_t)A.tri_blocks, s);
    // the initial state is the equilibrium of the current frame 0
    if (e == cudaSuccess) e = iblb::launch_init(lb->v, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint set-up");

    const int readout = m->readout_every;
    void *rec_saved = lb->v.rec;
    std::vector<cudaGraphExec_t> graphs;  // destroyed on return (they hold workspace addresses)
    // Recording run of segment [t0, t0 + len): before each step, the node
    // positions r_t go to the trajectory slot (on the stream of the droplet
    // kernels, which wrote them) and the lattice records its moments into
    // the step's slot.  Full-length segments replay a captured graph (one
    // per t0 mod 6 -- parity and patch buffer -- and shape-record setting);
    // a shorter one runs eagerly.  Shape records are taken only in the
    // forward pass, never when a segment is recorded again.
    // slot set `set` (segment sg uses set sg % 2) holds step k's moments and
    // positions + patch
    auto rec_slot = [&](int set, int k) -> char * { return ws + A.rec + A.rec_step * ((size_t)set * A.kmax + k); };
    auto traj_slot = [&](int set, int k) -> char * {
        return ws + A.traj + A.traj_step * ((size_t)set * A.kmax + k);
    };
    std::map<int, cudaGraphExec_t> rec_graph;
    int hook_set = 0;
    // step k of a recording: its force/spread kernel copies r_k and the
    // step's patch into the trajectory slot, its lattice kernels store the
    // moments into the moment slot
    auto record_hook = [&](int k, cudaStream_t, cudaStream_t) -> int {
        char *slot = traj_slot(hook_set, k);
        m->v.rec_r = reinterpret_cast<double *>(slot);
        m->v.rec_ctl = reinterpret_cast<Ctl *>(slot + A.traj_ctl);
        lb->v.rec = rec_slot(hook_set, k);
        return IBL_OK;
    };
    auto end_recording = [&]() {
        lb->v.rec = rec_saved;
        m->v.rec_r = nullptr;
        m->v.rec_ctl = nullptr;
    };
    // graph of a full-length recording starting at t0 (captured on first use)
    auto record_graph = [&](long long t0, bool shape_records, int set, cudaGraphExec_t *out) -> int {
        const int key = (int)(t0 % 6) + (shape_records ? 6 : 0) + 12 * set;
        auto it = rec_graph.find(key);
        if (it == rec_graph.end()) {
            const long long saved = lb->host_step;
            lb->host_step = t0;
            hook_set = set;
            m->readout_every = shape_records ? readout : 0;
            cudaGraphExec_t g = nullptr;
            const int r = capture_steps(lb, K, true, record_hook, &g);
            end_recording();
            m->readout_every = readout;
            lb->host_step = saved;
            if (r != IBL_OK) return r;
            graphs.push_back(g);
            // move the graph's device upload off the first launch
            const cudaError_t eu = cudaGraphUpload(g, lb->cap_stream);
            if (eu != cudaSuccess) return cuda_fail(eu, "recording graph upload");
            it = rec_graph.emplace(key, g).first;
        }
        if (out) *out = it->second;
        return IBL_OK;
    };
    auto record_segment = [&](long long t0, int len, bool shape_records, int set, cudaStream_t q) -> int {
        int r = IBL_OK;
        if (len == K) {
            cudaGraphExec_t g = nullptr;
            r = record_graph(t0, shape_records, set, &g);
            if (r != IBL_OK) return r;
            const cudaError_t ee = cudaGraphLaunch(g, q);
            if (ee != cudaSuccess) return cuda_fail(ee, "recording graph launch");
            lb->host_step = t0 + len;
            return IBL_OK;
        }
        lb->host_step = t0;
        hook_set = set;
        m->readout_every = shape_records ? readout : 0;
        for (int k = 0; k < len && r == IBL_OK; ++k) {
            r = record_hook(k, q, q);
            if (r == IBL_OK) r = one_step(lb, true, q, q);
        }
        end_recording();
        m->readout_every = readout;
        return r;
    };
    // Reverse sweep of a recorded segment on two streams, as the forward
    // step: the helper stream (high priority) runs the interpolation
    // adjoint, the patch nodes and the surface adjoint, the main stream the
    // nodes outside the patch; step k's patch update waits for step k+1's
    // outside update and vice versa.  Full-length segments replay a captured
    // graph (one per slot set and parity of the adjoint buffer pair).
    int cur = 0;  // lam[cur] holds the adjoint of the populations of step t + 1
    cudaGraphExec_t rev_graph[4] = {nullptr, nullptr, nullptr, nullptr};
    // events: 0-3 the reverse chain inside a capture, 4-7 eager, 8-9 a
    // recorded set ready, 10-11 a set released by its reverse sweep, 12 start
    cudaEvent_t ev[13] = {};
    cudaStream_t s_rec = nullptr;  // stream of the recordings that overlap the reverse sweep
    for (int k = 0; k < 13 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_rec, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        if (s_rec) cudaStreamDestroy(s_rec);
        return cuda_fail(e, "adjoint events");
    }
    auto enqueue_reverse = [&](int len, int c0, int set, cudaStream_t sL, cudaStream_t sH,
                               bool capture) -> cudaError_t {
        cudaEvent_t *eN = capture ? ev : ev + 4, *eF = eN + 2;
        cudaError_t ee = join(sL, sH, capture ? lb->cFork : lb->evFork);
        int c = c0;
        for (int k = len - 1; k >= 0 && ee == cudaSuccess; --k) {
            const int p = k & 1;
            char *slot = traj_slot(set, k);
            MeshView Mt = m->v;
            Mt.r = reinterpret_cast<double *>(slot);
            const Ctl *pc = reinterpret_cast<const Ctl *>(slot + A.traj_ctl);
            const void *rec = rec_slot(set, k);
            ee = iblb::launch_adj_interp(lb->v, Mt, J, rec, sH, lb->hi_prio);
            if (ee == cudaSuccess && k < len - 1) ee = cudaStreamWaitEvent(sH, eF[p ^ 1], 0);
            if (ee == cudaSuccess) ee = iblb::launch_adj_near(lb->v, J, rec, lam[c], lam[c ^ 1], pc, k, sH, lb->hi_prio);
            if (ee == cudaSuccess) ee = cudaEventRecord(eN[p], sH);
            if (ee == cudaSuccess) ee = iblb::launch_adj_surface(lb->v, Mt, J, sH, lb->hi_prio);
            if (ee == cudaSuccess && k < len - 1) ee = cudaStreamWaitEvent(sL, eN[p ^ 1], 0);
            if (ee == cudaSuccess) ee = iblb::launch_adj_far(lb->v, J, rec, lam[c], lam[c ^ 1], pc, k, sL);
            if (ee == cudaSuccess) ee = cudaEventRecord(eF[p], sL);
            c ^= 1;
        }
        if (ee == cudaSuccess) ee = join(sH, sL, capture ? lb->cJoin : lb->evJoin);
        return ee;
    };
    // graph of a full-length reverse sweep for buffer parity c0 and slot set
    // `set` (captured on first use)
    auto reverse_graph = [&](int c0, int set) -> int {
        cudaGraphExec_t &g = rev_graph[c0 + 2 * set];
        if (g) return IBL_OK;
        cudaStream_t cL = lb->cap_stream, cH = lb->cap_helper;
        cudaError_t ee = cudaStreamBeginCapture(cL, cudaStreamCaptureModeThreadLocal);
        if (ee != cudaSuccess) return cuda_fail(ee, "begin capture");
        const cudaError_t e1 = enqueue_reverse(K, c0, set, cL, cH, true);
        cudaGraph_t gr = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cL, &gr);
        ee = e1 != cudaSuccess ? e1 : e2;
        if (ee == cudaSuccess) ee = cudaGraphInstantiateWithFlags(&g, gr, cudaGraphInstantiateFlagUseNodePriority);
        if (gr) cudaGraphDestroy(gr);
        if (ee != cudaSuccess) return cuda_fail(ee, "adjoint graph capture");
        graphs.push_back(g);
        ee = cudaGraphUpload(g, lb->cap_stream);
        if (ee != cudaSuccess) return cuda_fail(ee, "adjoint graph upload");
        return IBL_OK;
    };
    auto reverse_segment = [&](long long t0, int len, int set) -> int {
        cudaError_t ee = iblb::launch_adj_set_t0(J, t0, s);
        if (ee != cudaSuccess) return cuda_fail(ee, "adjoint segment start");
        if (len == K) {
            const int r = reverse_graph(cur, set);
            if (r != IBL_OK) return r;
            ee = cudaGraphLaunch(rev_graph[cur + 2 * set], s);
        } else {
            ee = enqueue_reverse(len, cur, set, s, lb->helper, false);
        }
        if (ee != cudaSuccess) return cuda_fail(ee, "adjoint step launch");
        cur ^= (len & 1);
        return IBL_OK;
    };

    // forward pass: checkpoints at the segment starts; the last segment is
    // recorded on the way, so it needs no recomputation
    const long long last = A.n_seg - 1;
    for (long long sg = 0; sg < A.n_seg && st == IBL_OK; ++sg) {
        e = adj_save(lb, A, ws, sg, s);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "checkpoint");
            break;
        }
        const int len = (int)std::min<long long>(K, n_steps - sg * K);
        if (sg < last) st = ibl_step(lb, len);
        else st = record_segment(sg * K, len, true, (int)(sg & 1), s);
    }
    if (st == IBL_OK) {
        e = adj_save(lb, A, ws, A.n_seg, s);
        // seed: D of the final mesh and dD/dr_T
        if (e == cudaSuccess) e = iblb::launch_adj_seed(m->v, J, s);
        // the recordings start after the forward pass
        if (e == cudaSuccess) e = cudaEventRecord(ev[12], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_rec, ev[12], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "adjoint seed");
    }
    // Capture every graph the sweep below will replay while the GPU runs the
    // forward pass just enqueued (capture and instantiation are host work).
    {
        int c = cur;
        for (long long sg = last; sg >= 0 && st == IBL_OK; --sg) {
            const int len = (int)std::min<long long>(K, n_steps - sg * K);
            if (len == K) st = reverse_graph(c, (int)(sg & 1));
            if (st == IBL_OK && sg >= 1) st = record_graph((sg - 1) * K, false, (int)((sg - 1) & 1), nullptr);
            c ^= (len & 1);
        }
    }
    // Reverse sweep, last segment first.  While segment sg is swept back on
    // the main stream, segment sg - 1 is restored from its checkpoint and
    // recorded on its own stream into the other slot set; it waits for the
    // sweep of sg + 1, which used that set.  Both chains are latency-bound,
    // so they share the GPU well.
    for (long long sg = last; sg >= 0 && st == IBL_OK; --sg) {
        const long long t0 = sg * K;
        const int len = (int)std::min<long long>(K, n_steps - t0);
        const int set = (int)(sg & 1);
        if (sg < last) {
            e = cudaStreamWaitEvent(s, ev[8 + set], 0);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "adjoint ordering");
                break;
            }
        }
        st = reverse_segment(t0, len, set);
        if (st != IBL_OK) break;
        e = cudaEventRecord(ev[10 + set], s);
        if (e == cudaSuccess && sg >= 1) {
            const long long prev = sg - 1;
            const int pset = (int)(prev & 1);
            if (sg + 1 <= last) e = cudaStreamWaitEvent(s_rec, ev[10 + pset], 0);
            if (e == cudaSuccess) e = adj_restore(lb, A, ws, prev, s_rec);
            if (e == cudaSuccess) {
                st = record_segment(prev * K, K, false, pset, s_rec);
                if (st != IBL_OK) break;
                e = cudaEventRecord(ev[8 + pset], s_rec);
            }
        }
        if (e != cudaSuccess) st = cuda_fail(e, "adjoint recording");
    }
    // the main stream resumes after every recording
    if (e == cudaSuccess) e = cudaEventRecord(ev[12], s_rec);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[12], 0);
    if (e != cudaSuccess && st == IBL_OK) st = cuda_fail(e, "adjoint join");
    end_recording();
    // the initial populations depend on frame 0
    if (st == IBL_OK) {
        e = iblb::launch_adj_init(lb->v, J, lam[cur], s);
        if (e == cudaSuccess) e = iblb::launch_adj_reduce(J, nf, s);
        if (e != cudaSuccess) st = cuda_fail(e, "adjoint initial state");
    }
    // leave the lattice and droplet at the final step, as ibl_step would
    if (st == IBL_OK) {
        e = adj_restore(lb, A, ws, A.n_seg, s);
        if (e != cudaSuccess) st = cuda_fail(e, "final state restore");
    }
    lb->host_step = n_steps;
    std::vector<double> acc(1 + 9 * (size_t)nf);
    double obs0 = 0.0;
    if (st == IBL_OK) {
        e = cudaMemcpyAsync(acc.data(), J.acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&obs0, J.obs, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && dD_dr0) e = cudaMemcpyAsync(dD_dr0, J.lam_r, A.r_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "adjoint readout");
    }
    const cudaError_t es2 = cudaStreamSynchronize(s);
    cudaStreamSynchronize(s_rec);
    for (cudaGraphExec_t g : graphs) cudaGraphExecDestroy(g);
    for (cudaEvent_t x : ev) cudaEventDestroy(x);
    cudaStreamDestroy(s_rec);
    if (st != IBL_OK) return st;
    if (es2 != cudaSuccess) return cuda_fail(es2, "adjoint synchronize");
    st = lb_status_from_device(lb);
    if (st != IBL_OK) return st;
    if (D) *D = obs0;
    if (dD_dsigma) *dD_dsigma = acc[0];
    if (dD_dA) std::memcpy(dD_dA, acc.data() + 1, sizeof(double) * 9 * (size_t)nf);
    return IBL_OK;
}

}  // extern "C"
