// Internal interface between the C-ABI host code (iblb_api.cpp) and the
// CUDA kernels (iblb_kernels.cu).  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/iblb.h"

namespace iblb {

// Device control block of one lattice (lives in the lattice workspace).
struct alignas(128) Ctl {
    long long step;              // steps completed (advanced by the lattice kernel)
    unsigned int obs_blocks_done; // last-block ticket of the shape-record kernel
    int n_part;                  // bounding-box rows left for the next force/spread kernel
    int err;                     // IBL_ERRBIT_* (sticky)
    int reg_iters;               // iterations of the latest regularisation
    int n_records;               // shape records written
    int frame;                   // frame index applied by the next step
    int patch_lo[4];             // droplet patch: lower corner (normalised into the box)
    int patch_ext[4];            // extent (hi - lo), -1 = empty
    unsigned long long pad1[8];
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
    void *f;            // [19][qs]
    void *force;        // [3][nodes]
    void *vel;          // [3][nodes]
    void *rec;          // [7][nodes] or null: drho, u, F
    const double *frames;
    const void *frames_t;  // the frames in the storage precision
    int n_frames;
    int n_hold;
    Ctl *ctl;
};

struct MeshView {
    int nv, nt;
    double sigma;
    double *r;          // [nv][3]
    double *fn;         // [nv][3] nodal forces of the last step
    double *tn;         // [nt][3] scaled triangle normals of the last step
    const int *tris;    // [nt][3]
    const int *n2t_ptr; // [nv+1]
    const int *n2t;     // [3 nt] entries 3*t + slot
    const int *nb_ptr;  // [nv+1]
    const int *nb_idx;  // [3 nt]
    double *s0, *s1, *s2;  // regularisation scratch, [nv][3] each
    double *part;          // per-block bounding-box partials of the interpolation kernel, [blocks][6]
    double *obs_part;      // per-block partial sums of the shape-record kernel, [kObsBlocksMax][11]
    ibl_observables *ring;
    int ring_cap;
};

struct RegParams {
    double alpha, gamma, tol;
    int max_iter;
    int plus_sign;
};

// Device tables of an ensemble step (all members advance together).
struct EnsembleView {
    const LbView *lv;        // [n] member lattices (device copy)
    const MeshView *mv;      // [n] member meshes (device copy)
    const int *lat_member;   // [lat_blocks] member of each lattice block
    const int *lat_start;    // [n+1] first lattice block of each member
    const int *node_member;  // [node_blocks]
    const int *node_start;   // [n+1]
    const int *tri_member;   // [tri_blocks]
    const int *tri_start;    // [n+1]
    int lat_blocks, node_blocks, tri_blocks;
    int precision;
};

constexpr int kRingCap = 4096;
constexpr int kObsBlocksMax = 304;

cudaError_t launch_init(const LbView &L, cudaStream_t s);
cudaError_t launch_lattice(const LbView &L, bool odd, bool record, cudaStream_t s);
cudaError_t launch_advance(const LbView &L, cudaStream_t s);
cudaError_t launch_convert_frames(const LbView &L, int k0, int k1, cudaStream_t s);
cudaError_t launch_spread(const LbView &L, const MeshView &M, cudaStream_t s);
cudaError_t launch_interp(const LbView &L, const MeshView &M, cudaStream_t s);
cudaError_t launch_regularize(const LbView &L, const MeshView &M, const RegParams &p, cudaStream_t s);
cudaError_t launch_observables(const LbView &L, const MeshView &M, cudaStream_t s);
cudaError_t launch_patch_from_mesh(const LbView &L, const MeshView &M, cudaStream_t s);
cudaError_t launch_ensemble_step(const EnsembleView &E, bool odd, cudaStream_t s);

// records a message for ibl_last_error() and returns `code` (iblb_api.cpp)
int iblb_set_error(int code, const char *msg);

// library velocity order (shared with the host code of the library only)
void velocity_table(int c[19][3], double w[19]);

}  // namespace iblb
