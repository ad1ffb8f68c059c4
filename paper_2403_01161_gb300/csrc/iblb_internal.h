// Internal interface between the C-ABI host code (iblb_api.cpp) and the
// CUDA kernels (iblb_kernels.cu, iblb_adjoint.cu).  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/iblb.h"

namespace iblb {

// Device control block of one lattice (lives in the lattice workspace).
// Patch buffers: step t uses buffer t % 3.  The force/spread kernel of step
// t writes buffer (t + 1) % 3 while the outside update of step t - 1 may
// still read buffer (t - 1) % 3, so three buffers are needed.
struct alignas(128) Ctl {
    long long step;              // steps completed (advanced by the lattice kernel)
    unsigned int obs_blocks_done; // last-block ticket of the shape-record kernel
    int n_part;                  // bounding-box rows left for the next force/spread kernel
    int err;                     // IBL_ERRBIT_* (sticky)
    int reg_iters;               // iterations of the latest regularisation
    int n_records;               // shape records written
    int frame_par[2];            // frame index applied by the next step of parity p (0 even, 1 odd)
    int reg_count;               // regularisations performed (scheduled checks that triggered)
    double mesh_q;               // mesh quality at the last scheduled check: max over triangles of longest/shortest edge
    unsigned int cen_ticket;     // last-block ticket of the force kernel's centre-of-mass reduction
    int pad0;
    double centre[3][4];         // re-centring: centre of the boundary field of step t in buffer t % 3
    int patch_lo[3][4];          // droplet patch of step t in buffer t % 3: lower corner (inside the box)
    int patch_ext[3][4];         // extent (hi - lo), -1 = empty
};

// Views handed to kernels by value.
struct LbView {
    int n[3];
    int bc[3];          // IBL_BC_*
    int nodes;
    long long qs;       // population stride in elements
    int precision;      // IBL_FP32_DEV / IBL_FP64
    int rule;           // IBL_EDGE_*
    double omega;       // 1 / tau
    float omega_f;
    float inv_nx;       // 1 / n[0] (rounded): row of a node within its z plane in the batched lattice kernel
    void *f;            // [19][qs]
    void *force;        // [nodes][4]: x, y, z, 0 (one 16-byte record per node in FP32)
    void *vel;          // [nodes][4]
    void *rec;          // [7][nodes] or null: drho, u, F
    const double *frames;
    const void *frames_t;  // the frames in the storage precision
    int n_frames;
    int n_hold;
    int recentre;       // 1: the boundary field is centred on the droplet's centre of mass (ctl->centre)
    int visc;           // 1: viscosity ratio chi != 1, relaxation omega_in at nodes inside the droplet
    double omega_in;    // 1 / tau_in, tau_in = 1/2 + chi (tau - 1/2)
    float omega_in_f;
    unsigned int *ind;  // [ceil(nodes / 4)] inside flags, one byte per node (set by the indicator kernel, cleared by the patch update)
    Ctl *ctl;
    int staged;         // outside / whole-box update: 0 one thread per node with direct loads (k_lattice), v > 0 the staged pipeline's launch shape v (k_lattice_staged)
    int stage_fault;    // tests only: the staged update's stages never complete (its waits run out: IBL_ETIMEOUT)
    int prefetch;       // 1: the direct outside update prefetches into L2 one resident wave ahead
};

struct MeshView {
    int nv, nt;
    double sigma;
    double *r;          // [nv][3]
    double *fn;         // [nv][3] nodal forces of the last step
    const int *tris;    // [nt][3]
    const int *n2t_ptr; // [nv+1]
    const int *n2t;     // [3 nt] entries 3*t + slot
    const int *nb_ptr;  // [nv+1]
    const int *nb_idx;  // [3 nt]
    double *s0, *s1, *s2;  // regularisation scratch, [nv][3] each
    double *tm;            // [nt][3] m_t = -sigma N_t / (2 |N_t|) at the current positions (ensemble: written by the batched triangle kernel, read by the batched force kernel)
    double *part;          // per-block bounding-box partials of the interpolation kernel, [blocks][6]
    double *cpart;         // re-centring: per-block volume and first moment, [kCentreBlocks][4]
    double *obs_part;      // per-block partial sums of the shape-record kernel, [kObsBlocksMax][11]
    ibl_observables *ring;
    int ring_cap;
    // Adjoint recording (null otherwise): the force/spread kernel of a step
    // copies the positions the step starts from to rec_r [nv][3] and the
    // step's patch (its buffer's patch_lo / patch_ext) to rec_ctl.
    double *rec_r = nullptr;
    Ctl *rec_ctl = nullptr;
};

struct RegParams {
    double alpha, gamma, tol;
    int max_iter;
    int plus_sign;
    double trigger;  // > 0: smooth only when the mesh quality exceeds it; 0: always
    int keep_volume; // rescale about the volume centroid to the volume enclosed before the smoothing
};

// An ensemble step launches each phase once per group of up to kGroup
// members; the group's views travel by value in the kernel parameters (read
// in constant space), the block -> member tables live in device memory.
constexpr int kGroup = 64;
struct LbGroup {
    LbView v[kGroup];
};
struct MeshGroup {
    MeshView v[kGroup];
};

// Launch shapes of the ensemble step, the candidates of ibl_ensemble_tune:
// shape k = 8 c + 4 p + 2 t + w takes w resident waves of blocks of L2
// prefetch distance and 128 (t = 0) or 256 (t = 1) threads per block in the
// batched lattice update (each block takes that many consecutive nodes of
// one z plane of one member); p = 0 keeps the droplet-side working set in
// L2 (evict_last, as the single droplet does), p = 1 uses the default
// policy; c = 1, 2, 3 caps the grids of the droplet-side kernels at 1, 2, 4
// blocks per SM (they then stride over their work), c = 0 launches one
// block per work unit.
constexpr int kEnsShapes = IBL_ENSEMBLE_SHAPES;
constexpr int ens_shape_waves(int k) { return k & 1; }
constexpr int ens_shape_threads(int k) { return (k & 2) ? 256 : 128; }
constexpr bool ens_shape_keep(int k) { return (k & 4) == 0; }
constexpr int ens_shape_cap(int k) { return (k >> 3) == 0 ? 0 : ((k >> 3) == 3 ? 4 : (k >> 3)); }
constexpr bool ens_shape_capped(int k) { return ens_shape_cap(k) > 0; }
constexpr int kEnsDefaultShape = 16;

struct EnsembleView {
    std::vector<LbView> lv;      // host copies of the member views
    std::vector<MeshView> mv;
    // lattice block tables, one per block size (index 0: 128 threads, 1: 256)
    const int *lat_member[2];    // [lat blocks] member of each lattice block (device)
    const int *lat_start_d[2];   // [n+1] first block of each member (device)
    std::vector<int> lat_start[2];  // host copies
    const int *node_member;      // [node blocks]
    const int *node_start_d;
    std::vector<int> node_start;
    int precision;
    int shape;                   // kEnsShapes index of the batched lattice launch
};

// Discrete adjoint of one step (device pointers in the adjoint workspace).
struct AdjView {
    void *lam_u;     // [nodes][4] adjoint of the lattice velocity seen by the interpolation (storage type); kept zero between steps
    void *lam_F;     // [nodes][4] adjoint of the Eulerian force (storage type)
    double *lam_r;   // [nv][3] adjoint of the node positions
    double *a_part;  // [n_frames][acc_blocks][9] per-block partial sums of dD/dA_k (block-private)
    double *s_part;  // [tri_blocks] per-block partial sums of dD/dsigma (block-private)
    int lat_blocks;  // blocks of the lattice adjoint grid (nodes outside the patch)
    int acc_blocks;  // partial-sum slots per frame: lat_blocks, then the patch kernel's blocks
    int tri_blocks;  // blocks of the triangle kernel
    long long *t0;   // first step of the segment being swept (device, set before each segment)
    double *acc;     // [1 + 9 n_frames] dD/dsigma, then dD/dA_k row-major (written by the final reduction)
    double *obs;     // [11] D and the adjoints of the volume sums of the readout
};

constexpr int kRingCap = 4096;
constexpr int kObsBlocksMax = 304;

cudaError_t launch_init(const LbView &L, cudaStream_t s);
cudaError_t launch_lattice(const LbView &L, bool odd, bool record, int mode, int pbuf, cudaStream_t s);
// Whether the staged outside update can run on this lattice (FP32, Zou-He
// walls on every axis, 16-byte aligned population arrays).
bool staged_ok(const LbView &L);
// Sets the shared-memory attributes of the staged kernels of launch shape
// `kind` on the current device (outside any stream capture).
cudaError_t staged_prepare(int kind);
constexpr int kStagedShapes = 2;
cudaError_t launch_near(const LbView &L, bool odd, bool record, int pbuf, cudaStream_t s, int prio = 0);
enum { LAUNCH_FULL = 0, LAUNCH_FAR = 1 };
cudaError_t launch_convert_frames(const LbView &L, int k0, int k1, cudaStream_t s);
cudaError_t launch_spread(const LbView &L, const MeshView &M, int next_buf, cudaStream_t s, int prio = 0);
cudaError_t launch_interp(const LbView &L, const MeshView &M, cudaStream_t s, int prio = 0);
// Lanes per mesh node in the forward force/spread and interpolation kernels
// (128-thread blocks); each lane takes every kFwdLanes-th incident triangle
// and 16 / kFwdLanes of the 16 (y, z) rows of the 4x4x4 stencil.
// (8 measured best at 128^3 against 4 and 16.)
constexpr int kFwdLanes = 8;
static_assert(kFwdLanes == 4 || kFwdLanes == 8 || kFwdLanes == 16, "lanes per mesh node");
constexpr int kFwdNodesPerBlock = 128 / kFwdLanes;
// re-centring: the droplet's centre of mass at the current positions into ctl->centre[buf]
constexpr int kCentreBlocks = 16;
cudaError_t launch_centre(const LbView &L, const MeshView &M, int buf, cudaStream_t s, int prio = 0);
// viscosity ratio: the inside flags of the patch nodes of step `buf` from the current positions
cudaError_t launch_indicator(const LbView &L, const MeshView &M, int buf, cudaStream_t s, int prio = 0);
cudaError_t launch_regularize(const LbView &L, const MeshView &M, const RegParams &p, int buf, cudaStream_t s,
                              int prio = 0);
cudaError_t launch_observables(const LbView &L, const MeshView &M, cudaStream_t s, int prio = 0);
cudaError_t launch_patch_from_mesh(const LbView &L, const MeshView &M, int buf, cudaStream_t s);
// Ensemble step phases (two streams, as the single droplet's step):
// helper stream: pre (centre, triangle moments, forces + spread of the next
// patch) then near (patch nodes, after the previous far update) then interp;
// bound stream: far (nodes outside each member's patch, closes each
// member's step, after the previous near update).
constexpr int kEnsNearBlocks = 48;  // blocks per member of the batched patch-node kernel
cudaError_t launch_ensemble_pre(const EnsembleView &E, long long step, cudaStream_t s, int prio);
cudaError_t launch_ensemble_near(const EnsembleView &E, long long step, cudaStream_t s, int prio);
cudaError_t launch_ensemble_far(const EnsembleView &E, long long step, cudaStream_t s);
cudaError_t launch_ensemble_interp(const EnsembleView &E, cudaStream_t s, int prio);
// the shape records of the members with due[k] != 0, one launch per group
cudaError_t launch_observables_batched(const EnsembleView &E, const std::vector<char> &due, cudaStream_t s, int prio);

// adjoint kernels (iblb_adjoint.cu); Mt.r holds the positions r_t of the
// step, pc the control block recorded before it (its patch)
constexpr int kAdjNearBlocks = 304;
cudaError_t launch_adj_seed(const MeshView &M, const AdjView &J, cudaStream_t s);
cudaError_t launch_adj_interp(const LbView &L, const MeshView &Mt, const AdjView &J, const void *rec, cudaStream_t s,
                              int prio);
cudaError_t launch_adj_near(const LbView &L, const AdjView &J, const void *rec, const void *lam_next, void *lam_cur,
                            const Ctl *pc, int k_in_segment, cudaStream_t s, int prio);
cudaError_t launch_adj_far(const LbView &L, const AdjView &J, const void *rec, const void *lam_next, void *lam_cur,
                           const Ctl *pc, int k_in_segment, cudaStream_t s);
cudaError_t launch_adj_surface(const LbView &L, const MeshView &Mt, const AdjView &J, cudaStream_t s, int prio);
cudaError_t launch_adj_set_t0(const AdjView &J, long long t0, cudaStream_t s);
cudaError_t launch_adj_init(const LbView &L, const AdjView &J, const void *lam0, cudaStream_t s);
cudaError_t launch_adj_reduce(const AdjView &J, int n_frames, cudaStream_t s);
void adj_grid(const LbView &L, int nt, int *lat_blocks, int *near_blocks, int *tri_blocks);

// records a message for ibl_last_error() and returns `code` (iblb_api.cpp)
int iblb_set_error(int code, const char *msg);

// library velocity order (shared with the host code of the library only)
void velocity_table(int c[19][3], double w[19]);

}  // namespace iblb
