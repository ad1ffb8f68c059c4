// iblb_adjoint.cu -- discrete adjoint of one IBLB droplet step and of the
// Taylor deformation readout (Sec. 2, Sec. 3.1).  The objective is the
// deformation D of the final mesh; the parameters are the surface tension
// sigma and the velocity-gradient frames A_k.
//
// The reverse step t takes lambda_f(t+1) (adjoint of the pre-collision
// populations of step t+1, natural layout [i][node]) and lambda_r(t+1)
// (adjoint of the node positions), plus the density, velocity and force of
// step t recorded by a forward recomputation, and produces lambda_f(t),
// lambda_r(t), and the sigma / A contributions:
//   1. interpolation + advection: lambda_u = spread of lambda_r, and the
//      derivative of the 4-point weights (phi') into lambda_r;
//   2. lattice: streaming reversed (gather lambda from x + c_i), the
//      transpose of the BGK + Guo collision with half-force moments, and the
//      transpose of the boundary rebuild (face, edge, corner), which also
//      yields d/du_w and hence d/dA;
//   3. spread and nodal forces, per triangle: lambda_F interpolated at the
//      three vertices (with its weight gradient), d/dsigma, the area Hessian
//      times lambda_F and the weight derivative of the spread, added to
//      lambda_r of the vertices.
// Populations and lattice fields keep the storage precision T; node
// quantities and everything accumulated over steps are FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <utility>

#include "iblb_internal.h"
#include "iblb_device.cuh"

namespace iblb {
namespace {

// phi'(x) of the Peskin 4-point stencil (derivative of Sec. 3.1's phi).
template <typename T>
__device__ __forceinline__ T peskin_dphi(T x)
{
    const T a = fabs(x);
    const T sg = x < T(0) ? T(-1) : T(1);
    if (a < T(1)) return sg * T(0.125) * (T(-2) + (T(2) - T(4) * a) / sqrt(T(1) + T(4) * a - T(4) * a * a));
    if (a < T(2)) return sg * T(0.125) * (T(-2) - (T(6) - T(4) * a) / sqrt(T(-7) + T(12) * a - T(4) * a * a));
    return T(0);
}

template <typename T>
__device__ __forceinline__ void stencil_weights_d(const NodeStencil &S, int b, int c, T w[4], T dw[4], T &wy, T &dwy,
                                                  T &wz, T &dwz)
{
    T fx, fy, fz;
    if constexpr (sizeof(T) == 8) {
        fx = S.frac[0];
        fy = S.frac[1];
        fz = S.frac[2];
    } else {
        fx = T(S.frac[0]);
        fy = T(S.frac[1]);
        fz = T(S.frac[2]);
    }
    for (int a = 0; a < 4; ++a) {
        w[a] = peskin_phi<T>(fx + T(1 - a));
        dw[a] = peskin_dphi<T>(fx + T(1 - a));
    }
    wy = peskin_phi<T>(fy + T(1 - b));
    dwy = peskin_dphi<T>(fy + T(1 - b));
    wz = peskin_phi<T>(fz + T(1 - c));
    dwz = peskin_dphi<T>(fz + T(1 - c));
}

// Transpose of a buried link's moving-wall share 3 w_j (c_j.u_w).
template <typename T, int J>
__device__ __forceinline__ void buried_wall_share_adjoint(T l, T (&luw)[3])
{
    if constexpr (cxf(J) != 0) luw[0] += T(3.0 * wgt(J)) * T(cxf(J)) * l;
    if constexpr (cyf(J) != 0) luw[1] += T(3.0 * wgt(J)) * T(cyf(J)) * l;
    if constexpr (czf(J) != 0) luw[2] += T(3.0 * wgt(J)) * T(czf(J)) * l;
}

// ---------------------------------------------------------------------------
// Transpose of the boundary rebuild.  lt: adjoint of the rebuilt populations
// (outputs), lin: adjoint of the streamed populations (inputs; unknown and
// overwritten inputs get 0), luw += adjoint of the wall velocity.
template <typename T, int SX, int SY, int SZ>
__device__ __forceinline__ void bc_adjoint(const T (&lt)[19], T (&lin)[19], T rho, const T (&uw)[3], int rule,
                                           T (&luw)[3])
{
    constexpr int NB = (SX != 0) + (SY != 0) + (SZ != 0);
    if constexpr (NB == 1) {
        constexpr int A = SX != 0 ? 0 : (SY != 0 ? 1 : 2);
        constexpr int SA = SX != 0 ? SX : (SY != 0 ? SY : SZ);
        const T un = T(SA) * uw[A];
        sfor<19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            lin[k] = (comp(k, A) * SA < 0) ? T(0) : lt[k];
        });
        T lrho = T(0);
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (comp(j, A) * SA < 0) {
                constexpr int i = opp(j);
                constexpr int tn = (c2(i) == 2) ? 1 : 0;
                T cu = T(0), tu = T(0);
                if constexpr (cxf(i) != 0) cu += T(cxf(i)) * uw[0];
                if constexpr (cyf(i) != 0) cu += T(cyf(i)) * uw[1];
                if constexpr (czf(i) != 0) cu += T(czf(i)) * uw[2];
                if constexpr (A != 0 && cxf(i) != 0) tu += T(cxf(i)) * uw[0];
                if constexpr (A != 1 && cyf(i) != 0) tu += T(cyf(i)) * uw[1];
                if constexpr (A != 2 && czf(i) != 0) tu += T(czf(i)) * uw[2];
                const T lj = lt[j];
                lin[i] += lj;
                // alpha_j = (2 - |t|) c_i.u/6 + t.u/3 multiplies rho
                lrho -= lj * (T(2 - tn) * T(1.0 / 6.0) * cu + T(1.0 / 3.0) * tu);
                // d alpha_j / du_w
                if constexpr (cxf(i) != 0)
                    luw[0] -= lj * rho * (T(2 - tn) * T(1.0 / 6.0) * T(cxf(i)) + (A != 0 ? T(1.0 / 3.0) * T(cxf(i)) : T(0)));
                if constexpr (cyf(i) != 0)
                    luw[1] -= lj * rho * (T(2 - tn) * T(1.0 / 6.0) * T(cyf(i)) + (A != 1 ? T(1.0 / 3.0) * T(cyf(i)) : T(0)));
                if constexpr (czf(i) != 0)
                    luw[2] -= lj * rho * (T(2 - tn) * T(1.0 / 6.0) * T(czf(i)) + (A != 2 ? T(1.0 / 3.0) * T(czf(i)) : T(0)));
                // tangential momentum correction: + 1/2 sum_k (t_i.c_k) f_k over in-plane k
                sfor<19>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    if constexpr (comp(k, A) == 0) {
                        constexpr int tc = (A != 0 ? cxf(i) * cxf(k) : 0) + (A != 1 ? cyf(i) * cyf(k) : 0) +
                                           (A != 2 ? czf(i) * czf(k) : 0);
                        if constexpr (tc != 0) lin[k] += T(0.5) * T(tc) * lj;
                    }
                });
            }
        });
        // rho = (sum_tan f + 2 sum_out f) / (1 + u_w.n_out)
        const T inv = T(1) / (T(1) + un);
        sfor<19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if constexpr (comp(k, A) == 0) lin[k] += lrho * inv;
            else if constexpr (comp(k, A) * SA > 0) lin[k] += T(2) * lrho * inv;
        });
        luw[A] -= lrho * rho * inv * T(SA);
    } else if constexpr (NB == 2) {
        constexpr int E = SX == 0 ? 0 : (SY == 0 ? 1 : 2);
        constexpr int PE = E + 1, ME = E + 10;
        const bool slip = (rule == IBL_EDGE_COUNTER_SLIP);
        T lfb = T(12) * lt[0];
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && unknown_dir<SX, SY, SZ>(opp(j))) {
                lfb += lt[j];
                if (slip) buried_wall_share_adjoint<T, j>(lt[j], luw);
            }
        });
        // adjoint of each non-buried value, including its share of f_b
        T lv[19];
        sfor<19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if constexpr (k != 0 && !(unknown_dir<SX, SY, SZ>(k) && unknown_dir<SX, SY, SZ>(opp(k))))
                lv[k] = lt[k] + lfb * T(1.0 / 22.0);
            else
                lv[k] = T(0);
        });
        sfor<19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            lin[k] = (k != 0 && !unknown_dir<SX, SY, SZ>(k)) ? lv[k] : T(0);
        });
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && !unknown_dir<SX, SY, SZ>(opp(j))) {
                constexpr int i = opp(j);
                lin[i] += lv[j];
                if constexpr (comp(i, E) != 0) {
                    const T q = (slip ? T(0.25) : T(-0.25)) * T(comp(i, E)) * lv[j];
                    lin[PE] += q;
                    lin[ME] -= q;
                }
                if (slip) {
                    if constexpr (cxf(i) != 0) luw[0] -= T(6.0 * wgt(i)) * T(cxf(i)) * lv[j];
                    if constexpr (cyf(i) != 0) luw[1] -= T(6.0 * wgt(i)) * T(cyf(i)) * lv[j];
                    if constexpr (czf(i) != 0) luw[2] -= T(6.0 * wgt(i)) * T(czf(i)) * lv[j];
                    if constexpr (comp(i, E) != 0) luw[E] -= T(1.0 / 12.0) * T(comp(i, E)) * lv[j];
                }
            }
        });
    } else if constexpr (NB == 3) {
        const bool wall = (rule == IBL_EDGE_COUNTER_SLIP);
        T lfb = T(12) * lt[0];
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            constexpr int cs = cxf(j) * SX + cyf(j) * SY + czf(j) * SZ;
            if constexpr (j != 0 && cs == 0) {
                lfb += lt[j];
                if (wall) buried_wall_share_adjoint<T, j>(lt[j], luw);
            }
        });
        T lv[19];
        sfor<19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            constexpr int cs = cxf(k) * SX + cyf(k) * SY + czf(k) * SZ;
            if constexpr (k != 0 && cs != 0)
                lv[k] = lt[k] + lfb * T(1.0 / 18.0);
            else
                lv[k] = T(0);
        });
        sfor<19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            lin[k] = (k != 0 && !unknown_dir<SX, SY, SZ>(k)) ? lv[k] : T(0);
        });
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            constexpr int cs = cxf(j) * SX + cyf(j) * SY + czf(j) * SZ;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && cs != 0) {
                constexpr int i = opp(j);
                lin[i] += lv[j];
                if (wall) {
                    if constexpr (cxf(i) != 0) luw[0] -= T(6.0 * wgt(i)) * T(cxf(i)) * lv[j];
                    if constexpr (cyf(i) != 0) luw[1] -= T(6.0 * wgt(i)) * T(cyf(i)) * lv[j];
                    if constexpr (czf(i) != 0) luw[2] -= T(6.0 * wgt(i)) * T(czf(i)) * lv[j];
                }
            }
        });
    }
}

template <typename T>
__device__ __forceinline__ void bc_adjoint_dispatch(const T (&lt)[19], T (&lin)[19], T rho, const T (&uw)[3], int rule,
                                                    T (&luw)[3], int code)
{
#define IBL_BCA_CASE(a, b, c)                                 \
    case (a + 1) + 3 * (b + 1) + 9 * (c + 1):                 \
        bc_adjoint<T, a, b, c>(lt, lin, rho, uw, rule, luw);  \
        break;
    switch (code) {
        IBL_BCA_CASE(-1, 0, 0) IBL_BCA_CASE(1, 0, 0) IBL_BCA_CASE(0, -1, 0) IBL_BCA_CASE(0, 1, 0)
        IBL_BCA_CASE(0, 0, -1) IBL_BCA_CASE(0, 0, 1)
        IBL_BCA_CASE(-1, -1, 0) IBL_BCA_CASE(1, -1, 0) IBL_BCA_CASE(-1, 1, 0) IBL_BCA_CASE(1, 1, 0)
        IBL_BCA_CASE(-1, 0, -1) IBL_BCA_CASE(1, 0, -1) IBL_BCA_CASE(-1, 0, 1) IBL_BCA_CASE(1, 0, 1)
        IBL_BCA_CASE(0, -1, -1) IBL_BCA_CASE(0, 1, -1) IBL_BCA_CASE(0, -1, 1) IBL_BCA_CASE(0, 1, 1)
        IBL_BCA_CASE(-1, -1, -1) IBL_BCA_CASE(1, -1, -1) IBL_BCA_CASE(-1, 1, -1) IBL_BCA_CASE(1, 1, -1)
        IBL_BCA_CASE(-1, -1, 1) IBL_BCA_CASE(1, -1, 1) IBL_BCA_CASE(-1, 1, 1) IBL_BCA_CASE(1, 1, 1)
        default: break;
    }
#undef IBL_BCA_CASE
}

// Block sum of a few values (blockDim.x * blockDim.y a multiple of 32, at
// most 256), added in FP64 by threads 0..K-1 to the block's own slot
// dst[0..K-1].  Each slot belongs to one block of one grid shape, and
// launches on the stream are ordered, so no atomics are needed and the final
// sums do not depend on scheduling.
template <int K, typename V>
__device__ __forceinline__ void block_accumulate(V (&v)[K], double *dst)
{
    __shared__ V sh[8][K];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < K; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (tid < K) {
        V s = V(0);
        for (int w = 0; w < nw; ++w) s += sh[w][tid];
        dst[tid] += (double)s;
    }
}

__device__ __forceinline__ int lattice_block_index()
{
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// ---------------------------------------------------------------------------
// 2. lattice adjoint of node (x, y, z).  Nodes outside the droplet patch of
// the step (FAR) have no force and are not read by the interpolation, so
// their force and velocity adjoints are neither read nor written; patch
// nodes (NEAR) take the full transpose.  luwx accumulates the node's
// d/dA contribution (boundary nodes only).
enum { ADJ_FAR = 1, ADJ_NEAR = 2 };

template <typename T, int MODE>
__device__ __forceinline__ bool adj_node(const LbView &L, const AdjView &J, const int x, const int y, const int z,
                                         const T *__restrict__ rec, const T *__restrict__ lam_next,
                                         T *__restrict__ lam_cur, const int frame, T (&luwx)[9])
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int nxy = nx * ny, nodes = L.nodes;
    const int node = x + nx * y + nxy * z;
    const bool px = L.bc[0] == IBL_BC_PERIODIC, py = L.bc[1] == IBL_BC_PERIODIC, pz = L.bc[2] == IBL_BC_PERIODIC;
    const int sx = px ? 0 : (x == 0 ? -1 : (x == nx - 1 ? 1 : 0));
    const int sy = py ? 0 : (y == 0 ? -1 : (y == ny - 1 ? 1 : 0));
    const int sz = pz ? 0 : (z == 0 ? -1 : (z == nz - 1 ? 1 : 0));
    int oxm = -1, oxp = 1, oym = -nx, oyp = nx, ozm = -nxy, ozp = nxy;
    int miss = 0;
    if (x == 0) { if (px) oxm = nx - 1; else miss |= 1; }
    if (x == nx - 1) { if (px) oxp = -(nx - 1); else miss |= 2; }
    if (y == 0) { if (py) oym = (ny - 1) * nx; else miss |= 4; }
    if (y == ny - 1) { if (py) oyp = -(ny - 1) * nx; else miss |= 8; }
    if (z == 0) { if (pz) ozm = (nz - 1) * nxy; else miss |= 16; }
    if (z == nz - 1) { if (pz) ozp = -(nz - 1) * nxy; else miss |= 32; }
    // streaming reversed: the post-collision f_i(x) became f_i(x + c_i)
    T ls[19];
    sfor<19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cxf(i), cy = cyf(i), cz = czf(i);
        constexpr int need = (cx > 0 ? 2 : (cx < 0 ? 1 : 0)) | (cy > 0 ? 8 : (cy < 0 ? 4 : 0)) |
                             (cz > 0 ? 32 : (cz < 0 ? 16 : 0));
        const int off = (cx > 0 ? oxp : (cx < 0 ? oxm : 0)) + (cy > 0 ? oyp : (cy < 0 ? oym : 0)) +
                        (cz > 0 ? ozp : (cz < 0 ? ozm : 0));
        ls[i] = (miss & need) == 0 ? lam_next[i * nodes + node + off] : T(0);
    });
    const T drho = rec[node];
    const T ux = rec[nodes + node], uy = rec[2 * nodes + node], uz = rec[3 * nodes + node];
    T Fx = T(0), Fy = T(0), Fz = T(0), lux = T(0), luy = T(0), luz = T(0);
    if constexpr (MODE == ADJ_NEAR) {
        Fx = rec[4 * nodes + node];
        Fy = rec[5 * nodes + node];
        Fz = rec[6 * nodes + node];
        T *lu = static_cast<T *>(J.lam_u);  // [nodes][4]
        rec_ld3(lu + 4 * node, lux, luy, luz);
        if (lux != T(0) || luy != T(0) || luz != T(0)) rec_st3(lu + 4 * node, T(0), T(0), T(0));
    }
    const T rho = T(1) + drho;
    const T om = sizeof(T) == 4 ? T(L.omega_f) : T(L.omega);
    const T fpre = T(1) - T(0.5) * om;
    const T uu = ux * ux + uy * uy + uz * uz;
    // sums over lambda_i w_i (...)
    T P0 = 0, P1x = 0, P1y = 0, P1z = 0, P2x = 0, P2y = 0, P2z = 0, P3x = 0, P3y = 0, P3z = 0, Qcu = 0, Qcu2 = 0;
    sfor<19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const T lw = T(wgt(i)) * ls[i];
        T cu = T(0), cF = T(0);
        if constexpr (cxf(i) != 0) { cu += T(cxf(i)) * ux; cF += T(cxf(i)) * Fx; }
        if constexpr (cyf(i) != 0) { cu += T(cyf(i)) * uy; cF += T(cyf(i)) * Fy; }
        if constexpr (czf(i) != 0) { cu += T(czf(i)) * uz; cF += T(czf(i)) * Fz; }
        P0 += lw;
        Qcu += lw * cu;
        Qcu2 += lw * cu * cu;
        if constexpr (cxf(i) != 0) { P1x += T(cxf(i)) * lw; P2x += T(cxf(i)) * lw * cu; P3x += T(cxf(i)) * lw * cF; }
        if constexpr (cyf(i) != 0) { P1y += T(cyf(i)) * lw; P2y += T(cyf(i)) * lw * cu; P3y += T(cyf(i)) * lw * cF; }
        if constexpr (czf(i) != 0) { P1z += T(czf(i)) * lw; P2z += T(czf(i)) * lw * cu; P3z += T(czf(i)) * lw * cF; }
    });
    // f*_i = (1-om) f_i + om feq_i(rho, u) + S_i(u, F); u = (j + F/2)/rho
    const T orho = om * rho;
    const T Lrho = om * (P0 * (T(1) - T(1.5) * uu) + T(3) * Qcu + T(4.5) * Qcu2);
    const T Lux = lux + T(3) * orho * P1x + T(9) * orho * P2x - T(3) * (orho * ux + fpre * Fx) * P0 + T(9) * fpre * P3x;
    const T Luy = luy + T(3) * orho * P1y + T(9) * orho * P2y - T(3) * (orho * uy + fpre * Fy) * P0 + T(9) * fpre * P3y;
    const T Luz = luz + T(3) * orho * P1z + T(9) * orho * P2z - T(3) * (orho * uz + fpre * Fz) * P0 + T(9) * fpre * P3z;
    const T ir = T(1) / rho;
    if constexpr (MODE == ADJ_NEAR) {
        T *lF = static_cast<T *>(J.lam_F);  // [nodes][4]
        rec_st3(lF + 4 * node, fpre * (T(3) * P1x - T(3) * ux * P0 + T(9) * P2x) + T(0.5) * Lux * ir,
                fpre * (T(3) * P1y - T(3) * uy * P0 + T(9) * P2y) + T(0.5) * Luy * ir,
                fpre * (T(3) * P1z - T(3) * uz * P0 + T(9) * P2z) + T(0.5) * Luz * ir);
    }
    T lt[19];
    const T base = Lrho - (Lux * ux + Luy * uy + Luz * uz) * ir;
    sfor<19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        T v = (T(1) - om) * ls[i] + base;
        if constexpr (cxf(i) != 0) v += T(cxf(i)) * Lux * ir;
        if constexpr (cyf(i) != 0) v += T(cyf(i)) * Luy * ir;
        if constexpr (czf(i) != 0) v += T(czf(i)) * Luz * ir;
        lt[i] = v;
    });
    if (sx | sy | sz) {
        const T *A = static_cast<const T *>(L.frames_t) + 9 * frame;
        const T lx = T(x) - T(0.5) * T(nx - 1), ly = T(y) - T(0.5) * T(ny - 1), lz = T(z) - T(0.5) * T(nz - 1);
        const T uw[3] = {A[0] * lx + A[1] * ly + A[2] * lz, A[3] * lx + A[4] * ly + A[5] * lz,
                         A[6] * lx + A[7] * ly + A[8] * lz};
        T lin[19];
        T luw[3] = {T(0), T(0), T(0)};
        bc_adjoint_dispatch<T>(lt, lin, rho, uw, L.rule, luw, (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1));
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            lam_cur[i * nodes + node] = lin[i];
        });
        const T l[3] = {lx, ly, lz};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) luwx[3 * a + b] += luw[a] * l[b];
        return true;
    }
    sfor<19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        lam_cur[i * nodes + node] = lt[i];
    });
    return false;
}

// Step t = segment start (device) + k; its frame (held n_hold steps each)
// and its patch buffer t % 3 in the control block recorded before the step.
__device__ __forceinline__ void adj_step_of(const LbView &L, const AdjView &J, int k, int &frame, int &pbuf)
{
    const long long t = *J.t0 + k;
    const long long kf = t / L.n_hold;
    frame = (int)(kf < L.n_frames - 1 ? kf : L.n_frames - 1);
    pbuf = (int)(t % 3);
}

// Nodes outside the patch; partial sums in the slots of the lattice grid.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_lattice_far(LbView L, AdjView J, const T *__restrict__ rec,
                                                         const T *__restrict__ lam_next, T *__restrict__ lam_cur,
                                                         const Ctl *__restrict__ pc, int k_in_segment)
{
    int frame, pbuf;
    adj_step_of(L, J, k_in_segment, frame, pbuf);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    T luwx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool bnd = false;
    if (x < L.n[0] && y < L.n[1] && !node_in_patch(L, pc, pbuf, x, y, z))
        bnd = adj_node<T, ADJ_FAR>(L, J, x, y, z, rec, lam_next, lam_cur, frame, luwx);
    // blocks without boundary nodes have nothing to add (block-uniform test)
    if (__syncthreads_or(bnd))
        block_accumulate<9, T>(luwx, J.a_part + 9 * ((size_t)frame * J.acc_blocks + lattice_block_index()));
}

// Patch nodes (grid-stride over the patch box, x fastest); partial sums in
// the slots after the lattice grid's.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_lattice_near(LbView L, AdjView J, const T *__restrict__ rec,
                                                          const T *__restrict__ lam_next, T *__restrict__ lam_cur,
                                                          const Ctl *__restrict__ pc, int k_in_segment)
{
    int frame, buf;
    adj_step_of(L, J, k_in_segment, frame, buf);
    const int ex = pc->patch_ext[buf][0] + 1, ey = pc->patch_ext[buf][1] + 1, ez = pc->patch_ext[buf][2] + 1;
    const int lx = pc->patch_lo[buf][0], ly = pc->patch_lo[buf][1], lz = pc->patch_lo[buf][2];
    const int count = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
    T luwx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool bnd = false;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += gridDim.x * blockDim.x) {
        const int qz = idx / (ex * ey);
        const int rem = idx - qz * ex * ey;
        const int qy = rem / ex;
        const int qx = rem - qy * ex;
        int x = lx + qx, y = ly + qy, z = lz + qz;
        if (x >= L.n[0]) x -= L.n[0];  // a periodic patch may wrap once
        if (y >= L.n[1]) y -= L.n[1];
        if (z >= L.n[2]) z -= L.n[2];
        bnd |= adj_node<T, ADJ_NEAR>(L, J, x, y, z, rec, lam_next, lam_cur, frame, luwx);
    }
    if (__syncthreads_or(bnd))
        block_accumulate<9, T>(luwx,
                               J.a_part + 9 * ((size_t)frame * J.acc_blocks + J.lat_blocks + blockIdx.x));
}

// ---------------------------------------------------------------------------
// 1. interpolation + advection adjoint, 16 lanes per Lagrangian node.
template <typename T>
__global__ void __launch_bounds__(128) k_adj_interp(LbView L, MeshView M, AdjView J, const T *__restrict__ rec)
{
    const int gid = blockIdx.x * (kIbThreads / kLanesPerNode) + threadIdx.x / kLanesPerNode;
    const int lane = threadIdx.x % kLanesPerNode;
    const bool valid = gid < M.nv;
    const int i = valid ? gid : M.nv - 1;
    const NodeStencil S = node_stencil(L, M.r + 3 * i, lane);
    const double lr[3] = {J.lam_r[3 * i], J.lam_r[3 * i + 1], J.lam_r[3 * i + 2]};
    T g[3] = {T(0), T(0), T(0)};
    if (valid && S.ok) {
        const bool perx = L.bc[0] == IBL_BC_PERIODIC, pery = L.bc[1] == IBL_BC_PERIODIC,
                   perz = L.bc[2] == IBL_BC_PERIODIC;
        const int b = lane & 3, c = lane >> 2;
        T w[4], dw[4], wy, dwy, wz, dwz;
        stencil_weights_d<T>(S, b, c, w, dw, wy, dwy, wz, dwz);
        const int nx = L.n[0], nxy = L.n[0] * L.n[1], nodes = L.nodes;
        const int row = wrap_index(S.base[1] + b, L.n[1], pery) * nx + wrap_index(S.base[2] + c, L.n[2], perz) * nxy;
        T *lu = static_cast<T *>(J.lam_u);  // [nodes][4]
        const T lrx = T(lr[0]), lry = T(lr[1]), lrz = T(lr[2]);
        for (int a = 0; a < 4; ++a) {
            const int id = row + wrap_index(S.base[0] + a, nx, perx);
            const T dl = w[a] * wy * wz;
            rec_red3(lu + 4 * id, lrx * dl, lry * dl, lrz * dl);
            const T ul = rec[nodes + id] * lrx + rec[2 * nodes + id] * lry + rec[3 * nodes + id] * lrz;
            g[0] += ul * (dw[a] * wy * wz);
            g[1] += ul * (w[a] * dwy * wz);
            g[2] += ul * (w[a] * wy * dwz);
        }
    }
    for (int o = kLanesPerNode / 2; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) g[a] += __shfl_xor_sync(0xffffffffu, g[a], o, kLanesPerNode);
    if (valid && lane == 0)
        for (int a = 0; a < 3; ++a) J.lam_r[3 * i + a] = lr[a] + (double)g[a];
}

// 3. spread + nodal forces, 16 lanes per triangle t with vertices x_0..x_2
// (positions r_t).  Forward: F_k = sum over the triangles around vertex k of
// m_t x d_k (d_k = x_{k+2} - x_{k+1}, m_t = -sigma/2 n, n = N/|N|), spread
// as F_k Delta(x - x_k).  With l_k = sum_x lambda_F(x) Delta(x - x_k) and
// G_k = sum_x lambda_F(x) (grad_r Delta(x - x_k))^T, the triangle's share of
// sum_k l_k . F_k is m_t . W with W = sum_k d_k x l_k, so
//   d/dsigma       += -1/2 n . W,
//   d/dx_k (n . W) = (x_{k+1} - x_{k+2}) x v + (l_{k+1} - l_{k+2}) x n,
//                    v = (W - n (n . W)) / |N|,
// and the weights contribute G_k^T (m_t x d_k).  The three vertex sums go to
// lambda_r by FP64 atomics.
template <typename T>
__global__ void __launch_bounds__(128) k_adj_surface(LbView L, MeshView M, AdjView J)
{
    const int gid = blockIdx.x * (kIbThreads / kLanesPerNode) + threadIdx.x / kLanesPerNode;
    const int lane = threadIdx.x % kLanesPerNode;
    const bool valid = gid < M.nt;
    const int t = valid ? gid : M.nt - 1;
    int vid[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) vid[k] = M.tris[3 * t + k];
    T lk[3][3], Gk[3][3][3];
    const bool perx = L.bc[0] == IBL_BC_PERIODIC, pery = L.bc[1] == IBL_BC_PERIODIC,
               perz = L.bc[2] == IBL_BC_PERIODIC;
    const int nx = L.n[0], nxy = L.n[0] * L.n[1], nodes = L.nodes;
    const T *lF = static_cast<const T *>(J.lam_F);
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            lk[k][c] = T(0);
            #pragma unroll
            for (int b = 0; b < 3; ++b) Gk[k][c][b] = T(0);
        }
        const NodeStencil S = node_stencil(L, M.r + 3 * vid[k], lane);
        if (valid && S.ok) {
            const int b = lane & 3, c = lane >> 2;
            T w[4], dw[4], wy, dwy, wz, dwz;
            stencil_weights_d<T>(S, b, c, w, dw, wy, dwy, wz, dwz);
            const int row =
                wrap_index(S.base[1] + b, L.n[1], pery) * nx + wrap_index(S.base[2] + c, L.n[2], perz) * nxy;
#pragma unroll
            for (int a4 = 0; a4 < 4; ++a4) {
                const int id = row + wrap_index(S.base[0] + a4, nx, perx);
                T f[3];
                rec_ld3(lF + 4 * id, f[0], f[1], f[2]);
                const T wt = w[a4] * wy * wz;
                const T g[3] = {dw[a4] * wy * wz, w[a4] * dwy * wz, w[a4] * wy * dwz};
                #pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    lk[k][cc] += f[cc] * wt;
                    #pragma unroll
                    for (int bb = 0; bb < 3; ++bb) Gk[k][cc][bb] += f[cc] * g[bb];
                }
            }
        }
    }
    for (int o = kLanesPerNode / 2; o > 0; o >>= 1)
        #pragma unroll
        for (int k = 0; k < 3; ++k)
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
                lk[k][c] += __shfl_xor_sync(0xffffffffu, lk[k][c], o, kLanesPerNode);
                #pragma unroll
                for (int b = 0; b < 3; ++b) Gk[k][c][b] += __shfl_xor_sync(0xffffffffu, Gk[k][c][b], o, kLanesPerNode);
            }
    // the triangle's tail in the storage type (FP64 positions differenced
    // first); the vertex sums go to lambda_r in FP64
    T ds[1] = {T(0)};
    if (valid && lane == 0) {
        double x0[3];
        T x[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) x0[c] = M.r[3 * vid[0] + c];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) x[k][c] = T(M.r[3 * vid[k] + c] - x0[c]);
        T e1[3], e2[3], N[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e1[c] = x[1][c] - x[0][c];
            e2[c] = x[2][c] - x[0][c];
        }
        cross3(e1, e2, N);
        const T inv = T(1) / sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        const T n[3] = {N[0] * inv, N[1] * inv, N[2] * inv};
        const T hs = T(-0.5) * T(M.sigma);
        const T m[3] = {hs * n[0], hs * n[1], hs * n[2]};
        T d[3][3], W[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int kp = (k + 1) % 3, km = (k + 2) % 3;
#pragma unroll
            for (int c = 0; c < 3; ++c) d[k][c] = x[km][c] - x[kp][c];
            T cr[3];
            cross3(d[k], lk[k], cr);
#pragma unroll
            for (int c = 0; c < 3; ++c) W[c] += cr[c];
        }
        const T nW = n[0] * W[0] + n[1] * W[1] + n[2] * W[2];
        ds[0] = T(-0.5) * nW;
        const T v[3] = {(W[0] - n[0] * nW) * inv, (W[1] - n[1] * nW) * inv, (W[2] - n[2] * nW) * inv};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int kp = (k + 1) % 3, km = (k + 2) % 3;
            const T dx[3] = {x[kp][0] - x[km][0], x[kp][1] - x[km][1], x[kp][2] - x[km][2]};
            const T dl[3] = {lk[kp][0] - lk[km][0], lk[kp][1] - lk[km][1], lk[kp][2] - lk[km][2]};
            T c1[3], c2v[3], f[3];
            cross3(dx, v, c1);
            cross3(dl, n, c2v);
            cross3(m, d[k], f);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                T gw = T(0);
#pragma unroll
                for (int c = 0; c < 3; ++c) gw += f[c] * Gk[k][c][b];
                atomicAdd(J.lam_r + 3 * vid[k] + b, (double)(hs * (c1[b] + c2v[b]) + gw));
            }
        }
    }
    block_accumulate<1, T>(ds, J.s_part + blockIdx.x);
}

// ---------------------------------------------------------------------------
// Readout adjoint (Sec. 2): D = (sqrt(l_max) - sqrt(l_min)) / (...) of
// S = 5 (M2 - first first^T / V) / V, with the tetrahedra sums V, first
// (= int x dV) and M2 (= int x x^T dV) relative to node 0 as in the forward
// readout.  Prep (one block): D and the adjoints of M2, first and V.
__global__ void __launch_bounds__(256) k_adj_obs_prep(MeshView M, AdjView J)
{
    __shared__ double sh11[8][11];
    const double ref[3] = {M.r[0], M.r[1], M.r[2]};
    double acc[11];
    for (int k = 0; k < 11; ++k) acc[k] = 0.0;
    for (int t = threadIdx.x; t < M.nt; t += blockDim.x) {
        double p[3][3];
        for (int v = 0; v < 3; ++v) {
            const int id = M.tris[3 * t + v];
            for (int a = 0; a < 3; ++a) p[v][a] = M.r[3 * id + a] - ref[a];
        }
        double bc[3];
        cross3(p[1], p[2], bc);
        const double vt = (p[0][0] * bc[0] + p[0][1] * bc[1] + p[0][2] * bc[2]) / 6.0;
        const double s[3] = {p[0][0] + p[1][0] + p[2][0], p[0][1] + p[1][1] + p[2][1], p[0][2] + p[1][2] + p[2][2]};
        acc[0] += vt;
        for (int a = 0; a < 3; ++a) acc[1 + a] += vt * s[a];
        double m[6] = {0, 0, 0, 0, 0, 0};
        for (int v = 0; v < 4; ++v) {
            const double *q = v < 3 ? p[v] : s;
            m[0] += q[0] * q[0];
            m[1] += q[1] * q[1];
            m[2] += q[2] * q[2];
            m[3] += q[0] * q[1];
            m[4] += q[0] * q[2];
            m[5] += q[1] * q[2];
        }
        for (int k = 0; k < 6; ++k) acc[4 + k] += vt * m[k];
    }
    block_sum<11>(acc, sh11);
    if (threadIdx.x != 0) return;
    const double V = acc[0];
    const double first[3] = {acc[1] / 4.0, acc[2] / 4.0, acc[3] / 4.0};
    double M2[3][3] = {{acc[4], acc[7], acc[8]}, {acc[7], acc[5], acc[9]}, {acc[8], acc[9], acc[6]}};
    double C[3][3], Sm[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            C[a][b] = M2[a][b] / 20.0 - first[a] * first[b] / V;
            Sm[a][b] = 5.0 * C[a][b] / V;
        }
    double lam[3], vec[3][3];
    jacobi3(Sm, lam, vec);
    int imax = 0, imin = 0;
    for (int k = 1; k < 3; ++k) {
        if (lam[k] > lam[imax]) imax = k;
        if (lam[k] < lam[imin]) imin = k;
    }
    const double p = sqrt(fmax(lam[imax], 0.0)), q = sqrt(fmax(lam[imin], 0.0));
    const double D = (p - q) / (p + q);
    const double dDlmax = q / (p * (p + q) * (p + q)), dDlmin = -p / (q * (p + q) * (p + q));
    double G[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            G[a][b] = dDlmax * vec[a][imax] * vec[b][imax] + dDlmin * vec[a][imin] * vec[b][imin];
    // S = 5 C / V, C = M2/20 - first first^T / V (first, M2 here unscaled sums)
    double gC[3][3], trGC = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            gC[a][b] = 5.0 * G[a][b] / V;
            trGC += G[a][b] * C[a][b];
        }
    double Gf[3] = {0, 0, 0}, fGf = 0.0;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) Gf[a] += gC[a][b] * first[b];
        fGf += first[a] * Gf[a];
    }
    double *o = J.obs;
    o[0] = D;
    // adjoints of the per-triangle sums: acc4..9 (M2 * 20), acc1..3 (first * 4), acc0 (V)
    o[1] = gC[0][0] / 20.0;
    o[2] = gC[1][1] / 20.0;
    o[3] = gC[2][2] / 20.0;
    o[4] = gC[0][1] / 20.0;
    o[5] = gC[0][2] / 20.0;
    o[6] = gC[1][2] / 20.0;
    for (int a = 0; a < 3; ++a) o[7 + a] = -2.0 * Gf[a] / V / 4.0;
    o[10] = fGf / (V * V) - 5.0 * trGC / (V * V);
}

// Per node: lambda_r = dD/dr by the chain rule through each incident
// tetrahedron (ref, a, b, c): h = gM2 : Q + gfirst . s + gV multiplies
// dvt; Q = aa^T + bb^T + cc^T + ss^T and s = a + b + c depend on a directly.
__global__ void __launch_bounds__(128) k_adj_obs_nodes(MeshView M, AdjView J)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M.nv) return;
    const double *o = J.obs;
    const double gM[3][3] = {{o[1], o[4], o[5]}, {o[4], o[2], o[6]}, {o[5], o[6], o[3]}};
    const double gf[3] = {o[7], o[8], o[9]};
    const double gV = o[10];
    const double ref[3] = {M.r[0], M.r[1], M.r[2]};
    double g[3] = {0.0, 0.0, 0.0};
    for (int k = M.n2t_ptr[i]; k < M.n2t_ptr[i + 1]; ++k) {
        const int e = M.n2t[k];
        const int t = e / 3, slot = e - 3 * t;
        double p[3][3];
        for (int v = 0; v < 3; ++v) {
            const int id = M.tris[3 * t + v];
            for (int a = 0; a < 3; ++a) p[v][a] = M.r[3 * id + a] - ref[a];
        }
        double bc[3];
        cross3(p[1], p[2], bc);
        const double vt = (p[0][0] * bc[0] + p[0][1] * bc[1] + p[0][2] * bc[2]) / 6.0;
        const double s[3] = {p[0][0] + p[1][0] + p[2][0], p[0][1] + p[1][1] + p[2][1], p[0][2] + p[1][2] + p[2][2]};
        double h = gV + gf[0] * s[0] + gf[1] * s[1] + gf[2] * s[2];
        for (int v = 0; v < 4; ++v) {
            const double *q = v < 3 ? p[v] : s;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) h += gM[a][b] * q[a] * q[b];
        }
        // d vt / d p[slot] = p[slot+1] x p[slot+2] / 6
        double dv[3];
        cross3(p[(slot + 1) % 3], p[(slot + 2) % 3], dv);
        for (int a = 0; a < 3; ++a) {
            double gq = 0.0;
            for (int b = 0; b < 3; ++b) gq += gM[a][b] * (p[slot][b] + s[b]);
            g[a] += h * dv[a] / 6.0 + vt * 2.0 * gq + vt * gf[a];
        }
    }
    for (int a = 0; a < 3; ++a) J.lam_r[3 * i + a] = g[a];
}

// Initial state f = f_eq(1, A_0 (x - c)): d/dA_0 += sum_i lambda_i dfeq_i/du
// (x - c)^T.  Same grid as the lattice adjoint (its partial-sum slots).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_init(LbView L, AdjView J, const T *__restrict__ lam0)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (x < nx && y < ny) {
        const int node = x + nx * (y + ny * z);
        const double *A = L.frames;
        const double l[3] = {x - 0.5 * (nx - 1), y - 0.5 * (ny - 1), z - 0.5 * (nz - 1)};
        const double u[3] = {A[0] * l[0] + A[1] * l[1] + A[2] * l[2], A[3] * l[0] + A[4] * l[1] + A[5] * l[2],
                             A[6] * l[0] + A[7] * l[1] + A[8] * l[2]};
        double g[3] = {0.0, 0.0, 0.0};
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const double li = (double)lam0[i * L.nodes + node] * wgt(i);
            const double cu = cxf(i) * u[0] + cyf(i) * u[1] + czf(i) * u[2];
            g[0] += li * (3.0 * cxf(i) + 9.0 * cu * cxf(i) - 3.0 * u[0]);
            g[1] += li * (3.0 * cyf(i) + 9.0 * cu * cyf(i) - 3.0 * u[1]);
            g[2] += li * (3.0 * czf(i) + 9.0 * cu * czf(i) - 3.0 * u[2]);
        });
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) v[3 * a + b] = g[a] * l[b];
    }
    block_accumulate<9, double>(v, J.a_part + 9 * (size_t)lattice_block_index());
}

// Final sums: block 0 dD/dsigma over the triangle blocks, block 1 + j entry
// j of dD/dA over the lattice and patch blocks.  Fixed order, so the result is
// reproducible bit for bit.
__global__ void __launch_bounds__(256) k_adj_reduce(AdjView J)
{
    __shared__ double sh[8][1];
    double s[1] = {0.0};
    if (blockIdx.x == 0) {
        for (int b = threadIdx.x; b < J.tri_blocks; b += blockDim.x) s[0] += J.s_part[b];
    } else {
        const int j = blockIdx.x - 1, k = j / 9, c = j - 9 * k;
        const double *p = J.a_part + 9 * (size_t)k * J.acc_blocks + c;
        for (int b = threadIdx.x; b < J.acc_blocks; b += blockDim.x) s[0] += p[9 * (size_t)b];
    }
    block_sum<1>(s, sh);
    if (threadIdx.x == 0) J.acc[blockIdx.x] = s[0];
}

}  // namespace

// ---------------------------------------------------------------------------
static inline unsigned nblocks(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// The lattice adjoint and the initial-state kernel share one grid shape.
static void adj_lattice_grid(const LbView &L, dim3 &g, dim3 &b)
{
    const int bx = L.n[0] >= 128 ? 128 : ((L.n[0] + 31) / 32) * 32;
    const int by = 256 / bx;
    b = dim3(bx, by, 1);
    g = dim3((L.n[0] + bx - 1) / bx, (L.n[1] + by - 1) / by, L.n[2]);
}

void adj_grid(const LbView &L, int nt, int *lat_blocks, int *near_blocks, int *tri_blocks)
{
    dim3 g, b;
    adj_lattice_grid(L, g, b);
    *lat_blocks = (int)(g.x * g.y * g.z);
    *near_blocks = kAdjNearBlocks;
    *tri_blocks = (int)nblocks((long long)nt * kLanesPerNode, kIbThreads);
}

cudaError_t launch_adj_interp(const LbView &L, const MeshView &Mt, const AdjView &J, const void *rec, cudaStream_t s,
                              int prio)
{
    const dim3 g(nblocks((long long)Mt.nv * kLanesPerNode, kIbThreads)), b(kIbThreads);
    if (L.precision == IBL_FP64) return launch_p(k_adj_interp<double>, g, b, s, prio, L, Mt, J, (const double *)rec);
    return launch_p(k_adj_interp<float>, g, b, s, prio, L, Mt, J, (const float *)rec);
}

cudaError_t launch_adj_near(const LbView &L, const AdjView &J, const void *rec, const void *lam_next, void *lam_cur,
                            const Ctl *pc, int k_in_segment, cudaStream_t s, int prio)
{
    const dim3 g(kAdjNearBlocks), b(256);
    if (L.precision == IBL_FP64)
        return launch_p(k_adj_lattice_near<double>, g, b, s, prio, L, J, (const double *)rec, (const double *)lam_next,
                        (double *)lam_cur, pc, k_in_segment);
    return launch_p(k_adj_lattice_near<float>, g, b, s, prio, L, J, (const float *)rec, (const float *)lam_next,
                    (float *)lam_cur, pc, k_in_segment);
}

cudaError_t launch_adj_far(const LbView &L, const AdjView &J, const void *rec, const void *lam_next, void *lam_cur,
                           const Ctl *pc, int k_in_segment, cudaStream_t s)
{
    dim3 g, b;
    adj_lattice_grid(L, g, b);
    if (L.precision == IBL_FP64)
        k_adj_lattice_far<double><<<g, b, 0, s>>>(L, J, (const double *)rec, (const double *)lam_next,
                                                  (double *)lam_cur, pc, k_in_segment);
    else
        k_adj_lattice_far<float><<<g, b, 0, s>>>(L, J, (const float *)rec, (const float *)lam_next, (float *)lam_cur,
                                                 pc, k_in_segment);
    return cudaGetLastError();
}

cudaError_t launch_adj_surface(const LbView &L, const MeshView &Mt, const AdjView &J, cudaStream_t s, int prio)
{
    const dim3 g(nblocks((long long)Mt.nt * kLanesPerNode, kIbThreads)), b(kIbThreads);
    if (L.precision == IBL_FP64) return launch_p(k_adj_surface<double>, g, b, s, prio, L, Mt, J);
    return launch_p(k_adj_surface<float>, g, b, s, prio, L, Mt, J);
}

__global__ void k_adj_set_t0(AdjView J, long long t0) { *J.t0 = t0; }

cudaError_t launch_adj_set_t0(const AdjView &J, long long t0, cudaStream_t s)
{
    k_adj_set_t0<<<1, 1, 0, s>>>(J, t0);
    return cudaGetLastError();
}

cudaError_t launch_adj_seed(const MeshView &M, const AdjView &J, cudaStream_t s)
{
    k_adj_obs_prep<<<1, 256, 0, s>>>(M, J);
    k_adj_obs_nodes<<<nblocks(M.nv, 128), 128, 0, s>>>(M, J);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const LbView &L, const AdjView &J, const void *lam0, cudaStream_t s)
{
    dim3 g, b;
    adj_lattice_grid(L, g, b);
    if (L.precision == IBL_FP64) k_adj_init<double><<<g, b, 0, s>>>(L, J, static_cast<const double *>(lam0));
    else k_adj_init<float><<<g, b, 0, s>>>(L, J, static_cast<const float *>(lam0));
    return cudaGetLastError();
}

cudaError_t launch_adj_reduce(const AdjView &J, int n_frames, cudaStream_t s)
{
    k_adj_reduce<<<1 + 9 * n_frames, 256, 0, s>>>(J);
    return cudaGetLastError();
}

}  // namespace iblb
