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
//   3. spread: lambda_F of each node by interpolation of lambda_F(x), and
//      the weight derivative into lambda_r;
//   4. nodal forces F = -sigma dA/dx: d/dsigma and the area Hessian times
//      lambda_F into lambda_r (per triangle, then gathered per node).
// Populations keep the storage precision T; everything accumulated over
// nodes or steps is FP64.
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
        const bool wall = (rule == IBL_EDGE_PAPER_PLUS_WALL);
        T lfb = T(12) * lt[0];
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && unknown_dir<SX, SY, SZ>(opp(j))) lfb += lt[j];
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
                    lin[PE] -= T(0.25) * T(comp(i, E)) * lv[j];
                    lin[ME] += T(0.25) * T(comp(i, E)) * lv[j];
                }
                if (wall) {
                    if constexpr (cxf(i) != 0) luw[0] -= T(6.0 * wgt(i)) * T(cxf(i)) * lv[j];
                    if constexpr (cyf(i) != 0) luw[1] -= T(6.0 * wgt(i)) * T(cyf(i)) * lv[j];
                    if constexpr (czf(i) != 0) luw[2] -= T(6.0 * wgt(i)) * T(czf(i)) * lv[j];
                }
            }
        });
    } else if constexpr (NB == 3) {
        const bool wall = (rule == IBL_EDGE_PAPER_PLUS_WALL);
        T lfb = T(12) * lt[0];
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            constexpr int cs = cxf(j) * SX + cyf(j) * SY + czf(j) * SZ;
            if constexpr (j != 0 && cs == 0) lfb += lt[j];
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

// Warp sum of a few doubles, then one atomic per value from lane 0.
template <int K>
__device__ __forceinline__ void warp_atomic_add(double (&v)[K], double *dst, unsigned active)
{
    if (!active) return;
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < K; ++k)
            if (v[k] != 0.0) atomicAdd(dst + k, v[k]);
}

// ---------------------------------------------------------------------------
// 2. lattice adjoint, one thread per node.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_lattice(LbView L, AdjView J, const T *__restrict__ rec,
                                                     const T *__restrict__ lam_next, T *__restrict__ lam_cur,
                                                     int frame)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    double luwx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool bnd = false;
    if (x < nx && y < ny) {
        const int nxy = nx * ny, nodes = L.nodes;
        const int node = x + nx * y + nxy * z;
        const bool px = L.bc[0] == IBL_BC_PERIODIC, py = L.bc[1] == IBL_BC_PERIODIC,
                   pz = L.bc[2] == IBL_BC_PERIODIC;
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
        const T Fx = rec[4 * nodes + node], Fy = rec[5 * nodes + node], Fz = rec[6 * nodes + node];
        T *lu = static_cast<T *>(J.lam_u);
        const T lux = lu[node], luy = lu[nodes + node], luz = lu[2 * nodes + node];
        if (lux != T(0) || luy != T(0) || luz != T(0)) {
            lu[node] = T(0);
            lu[nodes + node] = T(0);
            lu[2 * nodes + node] = T(0);
        }
        const T rho = T(1) + drho;
        const T om = sizeof(T) == 4 ? T(L.omega_f) : T(L.omega);
        const T fpre = T(1) - T(0.5) * om;
        const T uu = ux * ux + uy * uy + uz * uz;
        // sums over lambda_i w_i (...)
        T P0 = 0, P1x = 0, P1y = 0, P1z = 0, P2x = 0, P2y = 0, P2z = 0, P3x = 0, P3y = 0, P3z = 0, Qcu = 0,
          Qcu2 = 0;
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
        T *lF = static_cast<T *>(J.lam_F);
        lF[node] = fpre * (T(3) * P1x - T(3) * ux * P0 + T(9) * P2x) + T(0.5) * Lux * ir;
        lF[nodes + node] = fpre * (T(3) * P1y - T(3) * uy * P0 + T(9) * P2y) + T(0.5) * Luy * ir;
        lF[2 * nodes + node] = fpre * (T(3) * P1z - T(3) * uz * P0 + T(9) * P2z) + T(0.5) * Luz * ir;
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
            bnd = true;
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
            const double l[3] = {(double)lx, (double)ly, (double)lz};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) luwx[3 * a + b] = (double)luw[a] * l[b];
        } else {
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                lam_cur[i * nodes + node] = lt[i];
            });
        }
    }
    const unsigned any = __ballot_sync(0xffffffffu, bnd);
    warp_atomic_add<9>(luwx, J.acc + 1 + 9 * frame, any);
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
    double g[3] = {0.0, 0.0, 0.0};
    if (valid && S.ok) {
        const bool perx = L.bc[0] == IBL_BC_PERIODIC, pery = L.bc[1] == IBL_BC_PERIODIC,
                   perz = L.bc[2] == IBL_BC_PERIODIC;
        const int b = lane & 3, c = lane >> 2;
        T w[4], dw[4], wy, dwy, wz, dwz;
        stencil_weights_d<T>(S, b, c, w, dw, wy, dwy, wz, dwz);
        const int nx = L.n[0], nxy = L.n[0] * L.n[1], nodes = L.nodes;
        const int row = wrap_index(S.base[1] + b, L.n[1], pery) * nx + wrap_index(S.base[2] + c, L.n[2], perz) * nxy;
        T *lu = static_cast<T *>(J.lam_u);
        const T lrx = T(lr[0]), lry = T(lr[1]), lrz = T(lr[2]);
        for (int a = 0; a < 4; ++a) {
            const int id = row + wrap_index(S.base[0] + a, nx, perx);
            const T dl = w[a] * wy * wz;
            atomicAdd(lu + id, lrx * dl);
            atomicAdd(lu + nodes + id, lry * dl);
            atomicAdd(lu + 2 * nodes + id, lrz * dl);
            const double ul = (double)rec[nodes + id] * lr[0] + (double)rec[2 * nodes + id] * lr[1] +
                              (double)rec[3 * nodes + id] * lr[2];
            g[0] += ul * (double)(dw[a] * wy * wz);
            g[1] += ul * (double)(w[a] * dwy * wz);
            g[2] += ul * (double)(w[a] * wy * dwz);
        }
    }
    for (int o = kLanesPerNode / 2; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) g[a] += __shfl_xor_sync(0xffffffffu, g[a], o, kLanesPerNode);
    if (valid && lane == 0)
        for (int a = 0; a < 3; ++a) J.lam_r[3 * i + a] = lr[a] + g[a];
}

// Scaled triangle normals of r_t (the forward force kernel's first stage).
__global__ void __launch_bounds__(256) k_adj_normals(MeshView M) { tri_body(M, blockIdx.x * blockDim.x + threadIdx.x); }

// 3. spread adjoint: lambda_F of the node (interpolated lambda_F field) and
// the weight derivative; F_i gathered from the triangle normals of r_t.
template <typename T>
__global__ void __launch_bounds__(128) k_adj_spread(LbView L, MeshView M, AdjView J)
{
    const int gid = blockIdx.x * (kIbThreads / kLanesPerNode) + threadIdx.x / kLanesPerNode;
    const int lane = threadIdx.x % kLanesPerNode;
    const bool valid = gid < M.nv;
    const int i = valid ? gid : M.nv - 1;
    double F[3] = {0.0, 0.0, 0.0};
    for (int k = M.n2t_ptr[i] + lane; k < M.n2t_ptr[i + 1]; k += kLanesPerNode) {
        const int e = M.n2t[k];
        const int t = e / 3, slot = e - 3 * t;
        const int vp = M.tris[3 * t + (slot == 2 ? 0 : slot + 1)];
        const int vm = M.tris[3 * t + (slot == 0 ? 2 : slot - 1)];
        const double d[3] = {M.r[3 * vm] - M.r[3 * vp], M.r[3 * vm + 1] - M.r[3 * vp + 1],
                             M.r[3 * vm + 2] - M.r[3 * vp + 2]};
        const double m[3] = {M.tn[3 * t], M.tn[3 * t + 1], M.tn[3 * t + 2]};
        double gg[3];
        cross3(m, d, gg);
        for (int a = 0; a < 3; ++a) F[a] += gg[a];
    }
    for (int o = kLanesPerNode / 2; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) F[a] += __shfl_xor_sync(0xffffffffu, F[a], o, kLanesPerNode);
    const NodeStencil S = node_stencil(L, M.r + 3 * i, lane);
    double lf[3] = {0.0, 0.0, 0.0}, g[3] = {0.0, 0.0, 0.0};
    if (valid && S.ok) {
        const bool perx = L.bc[0] == IBL_BC_PERIODIC, pery = L.bc[1] == IBL_BC_PERIODIC,
                   perz = L.bc[2] == IBL_BC_PERIODIC;
        const int b = lane & 3, c = lane >> 2;
        T w[4], dw[4], wy, dwy, wz, dwz;
        stencil_weights_d<T>(S, b, c, w, dw, wy, dwy, wz, dwz);
        const int nx = L.n[0], nxy = L.n[0] * L.n[1], nodes = L.nodes;
        const int row = wrap_index(S.base[1] + b, L.n[1], pery) * nx + wrap_index(S.base[2] + c, L.n[2], perz) * nxy;
        const T *lF = static_cast<const T *>(J.lam_F);
        // the forward spread adds T(F) * weight
        const double Ft[3] = {(double)T(F[0]), (double)T(F[1]), (double)T(F[2])};
        for (int a = 0; a < 4; ++a) {
            const int id = row + wrap_index(S.base[0] + a, nx, perx);
            const double l0 = (double)lF[id], l1 = (double)lF[nodes + id], l2 = (double)lF[2 * nodes + id];
            const double dl = (double)(w[a] * wy * wz);
            lf[0] += l0 * dl;
            lf[1] += l1 * dl;
            lf[2] += l2 * dl;
            const double fl = Ft[0] * l0 + Ft[1] * l1 + Ft[2] * l2;
            g[0] += fl * (double)(dw[a] * wy * wz);
            g[1] += fl * (double)(w[a] * dwy * wz);
            g[2] += fl * (double)(w[a] * wy * dwz);
        }
    }
    for (int o = kLanesPerNode / 2; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) {
            lf[a] += __shfl_xor_sync(0xffffffffu, lf[a], o, kLanesPerNode);
            g[a] += __shfl_xor_sync(0xffffffffu, g[a], o, kLanesPerNode);
        }
    if (valid && lane == 0)
        for (int a = 0; a < 3; ++a) {
            J.lam_Fn[3 * i + a] = lf[a];
            J.lam_r[3 * i + a] += g[a];
        }
}

// 4a. per triangle: unit normal, 1/|N| and W = sum_k d_k x l_k (d_k = x_{k+2}
// - x_{k+1}, l_k = lambda_F of vertex k); the triangle's share of
// sum_i lambda_Fi . F_i is -sigma/2 n.W, so d/dsigma += -1/2 n.W.
__global__ void __launch_bounds__(256) k_adj_tri(MeshView M, AdjView J)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double ds = 0.0;
    if (t < M.nt) {
        const int v[3] = {M.tris[3 * t], M.tris[3 * t + 1], M.tris[3 * t + 2]};
        double x[3][3], l[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                x[k][a] = M.r[3 * v[k] + a];
                l[k][a] = J.lam_Fn[3 * v[k] + a];
            }
        double e1[3], e2[3], N[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = x[1][a] - x[0][a];
            e2[a] = x[2][a] - x[0][a];
        }
        cross3(e1, e2, N);
        const double inv = 1.0 / sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        const double n[3] = {N[0] * inv, N[1] * inv, N[2] * inv};
        double W[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k) {
            const int kp = (k + 1) % 3, km = (k + 2) % 3;
            const double d[3] = {x[km][0] - x[kp][0], x[km][1] - x[kp][1], x[km][2] - x[kp][2]};
            double c[3];
            cross3(d, l[k], c);
            for (int a = 0; a < 3; ++a) W[a] += c[a];
        }
        double *o = J.tri_w + 7 * t;
        o[0] = n[0];
        o[1] = n[1];
        o[2] = n[2];
        o[3] = inv;
        o[4] = W[0];
        o[5] = W[1];
        o[6] = W[2];
        ds = -0.5 * (n[0] * W[0] + n[1] * W[1] + n[2] * W[2]);
    }
    double v1[1] = {ds};
    warp_atomic_add<1>(v1, J.acc, 1u);
}

// 4b. per node: lambda_r += -sigma/2 sum_t [ (x_{j+1} - x_{j+2}) x v_t +
// (l_{j+1} - l_{j+2}) x n_t ],  v_t = (W - n (n.W)) / |N|,  j = slot of the node.
__global__ void __launch_bounds__(128) k_adj_force_nodes(MeshView M, AdjView J)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M.nv) return;
    double g[3] = {0.0, 0.0, 0.0};
    for (int k = M.n2t_ptr[i]; k < M.n2t_ptr[i + 1]; ++k) {
        const int e = M.n2t[k];
        const int t = e / 3, slot = e - 3 * t;
        const int vp = M.tris[3 * t + (slot + 1) % 3], vm = M.tris[3 * t + (slot + 2) % 3];
        const double *o = J.tri_w + 7 * t;
        const double n[3] = {o[0], o[1], o[2]};
        const double nW = n[0] * o[4] + n[1] * o[5] + n[2] * o[6];
        const double v[3] = {(o[4] - n[0] * nW) * o[3], (o[5] - n[1] * nW) * o[3], (o[6] - n[2] * nW) * o[3]};
        const double dx[3] = {M.r[3 * vp] - M.r[3 * vm], M.r[3 * vp + 1] - M.r[3 * vm + 1],
                              M.r[3 * vp + 2] - M.r[3 * vm + 2]};
        const double dl[3] = {J.lam_Fn[3 * vp] - J.lam_Fn[3 * vm], J.lam_Fn[3 * vp + 1] - J.lam_Fn[3 * vm + 1],
                              J.lam_Fn[3 * vp + 2] - J.lam_Fn[3 * vm + 2]};
        double c1[3], c2v[3];
        cross3(dx, v, c1);
        cross3(dl, n, c2v);
        for (int a = 0; a < 3; ++a) g[a] += c1[a] + c2v[a];
    }
    for (int a = 0; a < 3; ++a) J.lam_r[3 * i + a] += -0.5 * M.sigma * g[a];
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
// (x - c)^T.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_init(LbView L, AdjView J, const T *__restrict__ lam0)
{
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (node < L.nodes) {
        const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
        const int z = node / (nx * ny);
        const int rem = node - z * nx * ny;
        const int y = rem / nx;
        const int x = rem - y * nx;
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
    warp_atomic_add<9>(v, J.acc + 1, 1u);
}

}  // namespace

// ---------------------------------------------------------------------------
static inline unsigned nblocks(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_adj_step(const LbView &L, const MeshView &Mt, const AdjView &J, const void *rec, const void *lam_next,
                            void *lam_cur, int frame, cudaStream_t s)
{
    dim3 g, b;
    {
        const int bx = L.n[0] >= 128 ? 128 : ((L.n[0] + 31) / 32) * 32;
        const int by = 256 / bx;
        b = dim3(bx, by, 1);
        g = dim3((L.n[0] + bx - 1) / bx, (L.n[1] + by - 1) / by, L.n[2]);
    }
    const unsigned gn = nblocks((long long)Mt.nv * kLanesPerNode, kIbThreads);
    if (L.precision == IBL_FP64) {
        k_adj_interp<double><<<gn, kIbThreads, 0, s>>>(L, Mt, J, static_cast<const double *>(rec));
        k_adj_lattice<double><<<g, b, 0, s>>>(L, J, static_cast<const double *>(rec),
                                              static_cast<const double *>(lam_next), static_cast<double *>(lam_cur),
                                              frame);
    } else {
        k_adj_interp<float><<<gn, kIbThreads, 0, s>>>(L, Mt, J, static_cast<const float *>(rec));
        k_adj_lattice<float><<<g, b, 0, s>>>(L, J, static_cast<const float *>(rec),
                                             static_cast<const float *>(lam_next), static_cast<float *>(lam_cur), frame);
    }
    k_adj_normals<<<nblocks(Mt.nt, 256), 256, 0, s>>>(Mt);  // triangle normals of r_t for the nodal forces
    if (L.precision == IBL_FP64) k_adj_spread<double><<<gn, kIbThreads, 0, s>>>(L, Mt, J);
    else k_adj_spread<float><<<gn, kIbThreads, 0, s>>>(L, Mt, J);
    k_adj_tri<<<nblocks(Mt.nt, 256), 256, 0, s>>>(Mt, J);
    k_adj_force_nodes<<<nblocks(Mt.nv, 128), 128, 0, s>>>(Mt, J);
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
    if (L.precision == IBL_FP64) k_adj_init<double><<<nblocks(L.nodes, 256), 256, 0, s>>>(L, J, static_cast<const double *>(lam0));
    else k_adj_init<float><<<nblocks(L.nodes, 256), 256, 0, s>>>(L, J, static_cast<const float *>(lam0));
    return cudaGetLastError();
}

}  // namespace iblb
