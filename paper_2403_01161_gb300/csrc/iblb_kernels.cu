// iblb_kernels.cu -- sm_103a kernels of one IBLB droplet step
// (arXiv:2403.01161, Sec. 3.1-3.3).
//
// Lattice: D3Q19 populations stored in place with the AA access pattern as
// deviations g_i = f_i - w_i (rho_0 = 1), structure of arrays [19][qs] with
// x fastest.  An even step reads slot i of node x and writes the
// post-collision value back to slot opp(i) of the same node; an odd step
// reads slot opp(i) of node x - c_i and writes slot i of node x + c_i.  Wet
// boundary nodes rebuild the populations whose source lies outside the box
// on both parities (Zou-He face rule, edge and corner rules), and skip the
// loads and stores that would leave the box, so no halo is needed.
//
// Immersed boundary: node positions and nodal forces in FP64; the Eulerian
// force and velocity live in full-size arrays of the population type, but
// only the droplet patch (bounding box of the 4x4x4 stencils) is ever
// touched: the spread adds into it, the lattice kernel reads and re-zeroes it
// and stores the velocity there, the interpolation reads it.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <algorithm>
#include <mutex>
#include <set>
#include <type_traits>
#include <utility>

#include "iblb_internal.h"
#include "iblb_device.cuh"

namespace iblb {
namespace {

// Half of the moving-wall difference f_eq(c_j) - f_eq(-c_j) at rho0 = 1:
// 3 w_j (c_j.u_w).
template <typename T, int J>
__device__ __forceinline__ T buried_wall_share(const T (&uw)[3])
{
    T cu = T(0);
    if constexpr (cxf(J) != 0) cu += T(cxf(J)) * uw[0];
    if constexpr (cyf(J) != 0) cu += T(cyf(J)) * uw[1];
    if constexpr (czf(J) != 0) cu += T(czf(J)) * uw[2];
    return T(3.0 * wgt(J)) * cu;
}

template <typename T, int SX, int SY, int SZ>
__device__ __forceinline__ void bc_apply(T (&f)[19], const T (&uw)[3], int rule)
{
    constexpr int NB = (SX != 0) + (SY != 0) + (SZ != 0);
    if constexpr (NB == 1) {
        // Face, Eq. (ZH_bulk) with the Zou-He closure for the density.
        constexpr int A = SX != 0 ? 0 : (SY != 0 ? 1 : 2);
        constexpr int SA = SX != 0 ? SX : (SY != 0 ? SY : SZ);
        const T un = T(SA) * uw[A];
        T sum_tan = 0, sum_out = 0;
        T P[3] = {0, 0, 0};  // tangential momentum of the in-plane populations
        sfor<19>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if constexpr (comp(k, A) == 0) {
                sum_tan += f[k];
                if constexpr (cxf(k) != 0) P[0] += T(cxf(k)) * f[k];
                if constexpr (cyf(k) != 0) P[1] += T(cyf(k)) * f[k];
                if constexpr (czf(k) != 0) P[2] += T(czf(k)) * f[k];
            } else if constexpr (comp(k, A) * SA > 0) {
                sum_out += f[k];
            }
        });
        const T drho = (sum_tan + T(2) * sum_out - un) / (T(1) + un);
        const T rho = T(1) + drho;
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (comp(j, A) * SA < 0) {
                constexpr int i = opp(j);
                constexpr int tn = (c2(i) == 2) ? 1 : 0;  // |t_i| for t_i = c_i - (c_i.n)n
                T cu = T(0), tu = T(0), corr = T(0);
                if constexpr (cxf(i) != 0) cu += T(cxf(i)) * uw[0];
                if constexpr (cyf(i) != 0) cu += T(cyf(i)) * uw[1];
                if constexpr (czf(i) != 0) cu += T(czf(i)) * uw[2];
                if constexpr (A != 0 && cxf(i) != 0) { tu += T(cxf(i)) * uw[0]; corr += T(cxf(i)) * P[0]; }
                if constexpr (A != 1 && cyf(i) != 0) { tu += T(cyf(i)) * uw[1]; corr += T(cyf(i)) * P[1]; }
                if constexpr (A != 2 && czf(i) != 0) { tu += T(czf(i)) * uw[2]; corr += T(czf(i)) * P[2]; }
                f[j] = f[i] - T(2 - tn) * rho * T(1.0 / 6.0) * cu - rho * T(1.0 / 3.0) * tu + T(0.5) * corr;
            }
        });
    } else if constexpr (NB == 2) {
        // Edge, Eq. (ZH_edges) (t_i = projection of c_i on the edge line),
        // then the buried links, Eq. (zh-buried-links-edges), f_0 = 12 f_b.
        // Counter-slip reading (default): the tangential sum with the face
        // rule's sign, so that it cancels the edge-line momentum f_{+e} -
        // f_{-e}, moving-wall bounce-back, the wall's edge-line share
        // -(t_i.u_w)/12, and each buried link plus its half of the
        // moving-wall difference 3 w_j (c_j.u_w): the node then carries
        // exactly u_w (rho0 = 1).  The literal rule: the printed sign and no
        // wall terms.
        constexpr int E = SX == 0 ? 0 : (SY == 0 ? 1 : 2);
        constexpr int PE = E + 1, ME = E + 10;  // +e_E and -e_E in the library order
        static_assert(comp(PE, E) == 1 && comp(ME, E) == -1, "axis links");
        const T dE = f[PE] - f[ME];
        const bool slip = (rule == IBL_EDGE_COUNTER_SLIP);
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && !unknown_dir<SX, SY, SZ>(opp(j))) {
                constexpr int i = opp(j);
                T v = f[i];
                if constexpr (comp(i, E) != 0) v += (slip ? T(0.25) : T(-0.25)) * T(comp(i, E)) * dE;
                if (slip) {
                    T cu = T(0);
                    if constexpr (cxf(i) != 0) cu += T(cxf(i)) * uw[0];
                    if constexpr (cyf(i) != 0) cu += T(cyf(i)) * uw[1];
                    if constexpr (czf(i) != 0) cu += T(czf(i)) * uw[2];
                    v -= T(6.0 * wgt(i)) * cu;
                    if constexpr (comp(i, E) != 0) v -= T(1.0 / 12.0) * T(comp(i, E)) * uw[E];
                }
                f[j] = v;
            }
        });
        T sb = T(0);
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if constexpr (i != 0 && !(unknown_dir<SX, SY, SZ>(i) && unknown_dir<SX, SY, SZ>(opp(i)))) sb += f[i];
        });
        const T fb = sb * T(1.0 / 22.0);
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && unknown_dir<SX, SY, SZ>(opp(j)))
                f[j] = slip ? fb + buried_wall_share<T, j>(uw) : fb;
        });
        f[0] = T(12) * fb;
    } else if constexpr (NB == 3) {
        // Corner, Eq. (zh-buried-links-corners); non-buried unknowns take
        // (moving-wall) bounce-back, buried links (plus their moving-wall
        // share under the counter-slip reading); f_0 = 12 f_b.
        const bool wall = (rule == IBL_EDGE_COUNTER_SLIP);
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            constexpr int cs = -(cxf(j) * SX + cyf(j) * SY + czf(j) * SZ);
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && cs != 0) {
                constexpr int i = opp(j);
                T v = f[i];
                if (wall) {
                    T cu = T(0);
                    if constexpr (cxf(i) != 0) cu += T(cxf(i)) * uw[0];
                    if constexpr (cyf(i) != 0) cu += T(cyf(i)) * uw[1];
                    if constexpr (czf(i) != 0) cu += T(czf(i)) * uw[2];
                    v -= T(6.0 * wgt(i)) * cu;
                }
                f[j] = v;
            }
        });
        T sb = T(0);
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cs = cxf(i) * SX + cyf(i) * SY + czf(i) * SZ;
            if constexpr (i != 0 && cs != 0) sb += f[i];
        });
        const T fb = sb * T(1.0 / 18.0);
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            constexpr int cs = cxf(j) * SX + cyf(j) * SY + czf(j) * SZ;
            if constexpr (j != 0 && cs == 0) f[j] = wall ? fb + buried_wall_share<T, j>(uw) : fb;
        });
        f[0] = T(12) * fb;
    }
}

template <typename T>
__device__ __forceinline__ void bc_dispatch(T (&f)[19], const T (&uw)[3], int rule, int code)
{
#define IBL_BC_CASE(a, b, c)                              \
    case (a + 1) + 3 * (b + 1) + 9 * (c + 1):             \
        bc_apply<T, a, b, c>(f, uw, rule);                \
        break;
    switch (code) {
        IBL_BC_CASE(-1, 0, 0) IBL_BC_CASE(1, 0, 0) IBL_BC_CASE(0, -1, 0) IBL_BC_CASE(0, 1, 0)
        IBL_BC_CASE(0, 0, -1) IBL_BC_CASE(0, 0, 1)
        IBL_BC_CASE(-1, -1, 0) IBL_BC_CASE(1, -1, 0) IBL_BC_CASE(-1, 1, 0) IBL_BC_CASE(1, 1, 0)
        IBL_BC_CASE(-1, 0, -1) IBL_BC_CASE(1, 0, -1) IBL_BC_CASE(-1, 0, 1) IBL_BC_CASE(1, 0, 1)
        IBL_BC_CASE(0, -1, -1) IBL_BC_CASE(0, 1, -1) IBL_BC_CASE(0, -1, 1) IBL_BC_CASE(0, 1, 1)
        IBL_BC_CASE(-1, -1, -1) IBL_BC_CASE(1, -1, -1) IBL_BC_CASE(-1, 1, -1) IBL_BC_CASE(1, 1, -1)
        IBL_BC_CASE(-1, -1, 1) IBL_BC_CASE(1, -1, 1) IBL_BC_CASE(-1, 1, 1) IBL_BC_CASE(1, 1, 1)
        default: break;
    }
#undef IBL_BC_CASE
}

// ---------------------------------------------------------------------------
// Lattice update: streaming (AA pattern) + boundary rebuild + moments with
// half-force momentum + BGK + Guo source, Eqs. (LBMEQ)-(density_velocity_LB).
// One thread per node; blocks tile (x, y) rows of one z plane, so no index
// division is needed.  Indices are 32-bit (19 * stride < 2^31 is checked on
// the host).  The collision works on opposite pairs (c_i, -c_i), whose
// equilibrium and source terms share their even parts.
// Node sets of one lattice launch: every node, reading the droplet patch's
// force where the node lies in the patch (FULL); only the nodes outside the
// patch (FAR); only patch nodes (NEAR).  FAR and NEAR launches of the same
// step may run concurrently: in the AA pattern every population slot is read
// and written by one node only within a step.
enum { LAT_FULL = 0, LAT_FAR = 1, LAT_NEAR = 2 };

// 3 w_i, the weight of the odd (momentum) parts of the equilibrium and of
// the Guo source.  The exact values are 1/6 (|c_i|^2 = 1) and 1/12 (|c_i|^2
// = 2), and sum_i c_ia c_ia 3 w_i = 2/6 + 8/12 = 1 carries the momentum
// through the collision.  Rounded to nearest in FP32 both come out 2^-25
// relatively high, so that every collision would multiply the momentum by
// 1 + 3.0e-8 -- a bias that accumulates over the thousands of steps a
// velocity perturbation lives (L^2 / nu).  In FP32 1/6 is therefore rounded
// down instead (0x3E2AAAAA, 2^-24 relatively low), which makes
// 2 (3 w_1) + 8 (3 w_2) equal to 1 exactly; what remains of each product's
// error is its own rounding, without a common sign.
template <typename T, int i>
__device__ __forceinline__ T odd_weight()
{
    if constexpr (sizeof(T) == 4) return __int_as_float(c2(i) == 1 ? 0x3E2AAAAA : 0x3DAAAAAB);
    else return T(3.0 * wgt(i));
}

// The part of a node update after its 19 incoming populations g are in
// registers: boundary rebuild (sx, sy, sz: -1 / 0 / +1 where the node lies on
// a wall of that axis), patch force, moments, BGK + Guo, stores (AA pattern:
// even step own slots opp(i), odd step slot i at x + c_i), velocity record.
// Returns whether the node is unstable.
template <typename T, bool ODD, bool REC, int MODE, bool PER, class P = L2Keep>
__device__ __forceinline__ bool lattice_finish(const LbView &L, T (&g)[19], const int x, const int y, const int z,
                                               const int node, const bool in_patch, const int pbuf, const int sx,
                                               const int sy, const int sz)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int nxy = nx * ny;
    bool bad = false;
    {
        T *__restrict__ f = static_cast<T *>(L.f);
        struct NoKeep {};
        [[maybe_unused]] const std::conditional_t<MODE == LAT_NEAR, P, NoKeep> K;
        const int qs = (int)L.qs;
        const bool px = PER && L.bc[0] == IBL_BC_PERIODIC, py = PER && L.bc[1] == IBL_BC_PERIODIC,
                   pz = PER && L.bc[2] == IBL_BC_PERIODIC;
        if (sx | sy | sz) {
            // Eq. (velo_facce_cubo_da_gradiente) in the storage precision,
            // about the box centre or, with re-centring, about the droplet's
            // centre of mass at the start of the step (the offset in FP64)
            const T *A = static_cast<const T *>(L.frames_t) + 9 * L.ctl->frame_par[ODD ? 1 : 0];
            T lx, ly, lz;
            if (L.recentre) {
                const double *c = L.ctl->centre[pbuf];
                lx = T(double(x) - c[0]);
                ly = T(double(y) - c[1]);
                lz = T(double(z) - c[2]);
            } else {
                lx = T(x) - T(0.5) * T(nx - 1);
                ly = T(y) - T(0.5) * T(ny - 1);
                lz = T(z) - T(0.5) * T(nz - 1);
            }
            const T uw[3] = {A[0] * lx + A[1] * ly + A[2] * lz, A[3] * lx + A[4] * ly + A[5] * lz,
                             A[6] * lx + A[7] * ly + A[8] * lz};
            bc_dispatch<T>(g, uw, L.rule, (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1));
        }

        // droplet patch: read the spread force (and clear it), store u below;
        // both fields hold a 4-wide record (x, y, z, 0) per node
        T Fx = T(0), Fy = T(0), Fz = T(0);
        T *__restrict__ force = static_cast<T *>(L.force);
        if constexpr (MODE == LAT_NEAR) {
            K.ld3(force + 4 * node, Fx, Fy, Fz);
            K.st3(force + 4 * node, T(0), T(0), T(0));
        } else if (in_patch) {
            rec_ld3(force + 4 * node, Fx, Fy, Fz);
            rec_st3(force + 4 * node, T(0), T(0), T(0));
        }

        T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            drho += g[i];
            if constexpr (cxf(i) != 0) jx += T(cxf(i)) * g[i];
            if constexpr (cyf(i) != 0) jy += T(cyf(i)) * g[i];
            if constexpr (czf(i) != 0) jz += T(czf(i)) * g[i];
        });
        const T rho = T(1) + drho;
        const T ir = T(1) / rho;
        // rho u = j + F/2 (Eq. (density_velocity_LB)); the odd (momentum)
        // parts of the equilibrium are formed from it directly
        const T mx = jx + T(0.5) * Fx, my = jy + T(0.5) * Fy, mz = jz + T(0.5) * Fz;
        const T ux = mx * ir, uy = my * ir, uz = mz * ir;
        const T uu = ux * ux + uy * uy + uz * uz;
        bad = !(uu <= T(0.09)) || !(drho == drho);
        T om = sizeof(T) == 4 ? T(L.omega_f) : T(L.omega);
        if constexpr (MODE == LAT_NEAR) {
            // viscosity ratio: relaxation of the inside nodes (flags read and cleared)
            if (L.visc) {
                unsigned char *flag = reinterpret_cast<unsigned char *>(L.ind) + node;
                if (*flag) om = sizeof(T) == 4 ? T(L.omega_in_f) : T(L.omega_in);
                *flag = 0;
            }
        }
        const T fpre = T(1) - T(0.5) * om;
        const T uF = ux * Fx + uy * Fy + uz * Fz;
        const T dmr = drho - rho * (T(1.5) * uu);  // drho - (3/2) rho u.u
        {
            constexpr double w0 = wgt(0);
            const T geq = T(w0) * dmr;
            const T src = fpre * T(w0) * (T(-3) * uF);
            g[0] = g[0] + om * (geq - g[0]) + src;
        }
        sfor<9>([&](auto I) {
            constexpr int i = decltype(I)::value + 1;
            constexpr int j = opp(i);
            T cp = T(0), cF = T(0);  // c_i . rho u, c_i . F
            if constexpr (cxf(i) != 0) { cp += T(cxf(i)) * mx; cF += T(cxf(i)) * Fx; }
            if constexpr (cyf(i) != 0) { cp += T(cyf(i)) * my; cF += T(cyf(i)) * Fy; }
            if constexpr (czf(i) != 0) { cp += T(czf(i)) * mz; cF += T(czf(i)) * Fz; }
            const T cu = cp * ir;
            constexpr double w = wgt(i);
            const T w3 = odd_weight<T, i>();
            const T even_eq = T(w) * (T(4.5) * cp * cu + dmr);
            const T odd_eq = w3 * cp;
            const T even_src = fpre * T(w) * (T(9) * cu * cF - T(3) * uF);
            const T odd_src = fpre * w3 * cF;
            g[i] = g[i] + om * (even_eq + odd_eq - g[i]) + (even_src + odd_src);
            g[j] = g[j] + om * (even_eq - odd_eq - g[j]) + (even_src - odd_src);
        });

        if constexpr (!ODD) {
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                if constexpr (MODE == LAT_NEAR) K.st(f + opp(i) * qs + node, g[i]);
                else f[opp(i) * qs + node] = g[i];
            });
        } else {
            // destination x + c_i, slot i.  The node coordinates pass through
            // an opaque move, so the neighbour offsets are recomputed here
            // instead of being held in registers across the collision (which
            // made this kernel spill).
            int xs = x, ys = y, zs = z;
            asm volatile("mov.b32 %0, %0;" : "+r"(xs));
            asm volatile("mov.b32 %0, %0;" : "+r"(ys));
            asm volatile("mov.b32 %0, %0;" : "+r"(zs));
            const int nodes_ = xs + nx * ys + nxy * zs;
            int sxm = -1, sxp = 1, sym = -nx, syp = nx, szm = -nxy, szp = nxy, smiss = 0;
            if (xs == 0) { if (px) sxm = nx - 1; else smiss |= 1; }
            if (xs == nx - 1) { if (px) sxp = -(nx - 1); else smiss |= 2; }
            if (ys == 0) { if (py) sym = (ny - 1) * nx; else smiss |= 4; }
            if (ys == ny - 1) { if (py) syp = -(ny - 1) * nx; else smiss |= 8; }
            if (zs == 0) { if (pz) szm = (nz - 1) * nxy; else smiss |= 16; }
            if (zs == nz - 1) { if (pz) szp = -(nz - 1) * nxy; else smiss |= 32; }
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = cxf(i), cy = cyf(i), cz = czf(i);
                constexpr int need = (cx > 0 ? 2 : (cx < 0 ? 1 : 0)) | (cy > 0 ? 8 : (cy < 0 ? 4 : 0)) |
                                     (cz > 0 ? 32 : (cz < 0 ? 16 : 0));
                const int off = (cx > 0 ? sxp : (cx < 0 ? sxm : 0)) + (cy > 0 ? syp : (cy < 0 ? sym : 0)) +
                                (cz > 0 ? szp : (cz < 0 ? szm : 0));
                if ((smiss & need) == 0) {
                    if constexpr (MODE == LAT_NEAR) K.st(f + i * qs + nodes_ + off, g[i]);
                    else f[i * qs + nodes_ + off] = g[i];
                }
            });
        }
        if (in_patch) {
            T *__restrict__ vel = static_cast<T *>(L.vel);
            if constexpr (MODE == LAT_NEAR) K.st3(vel + 4 * node, ux, uy, uz);
            else rec_st3(vel + 4 * node, ux, uy, uz);
        }
        if constexpr (REC) {
            const int nodes = L.nodes;
            T *__restrict__ rec = static_cast<T *>(L.rec);
            rec[node] = drho;
            rec[nodes + node] = ux;
            rec[2 * nodes + node] = uy;
            rec[3 * nodes + node] = uz;
            rec[4 * nodes + node] = Fx;
            rec[5 * nodes + node] = Fy;
            rec[6 * nodes + node] = Fz;
        }
    }
    return bad;
}

// One node update with its loads from global memory.
// PER: some axis may be periodic (false: every axis has Zou-He walls, so
// the neighbour offsets are fixed and only the boundary tests remain).
// P: L2 policy of the patch nodes' accesses (LAT_NEAR).
template <typename T, bool ODD, bool REC, int MODE, bool PER, class P = L2Keep>
__device__ __forceinline__ bool lattice_node(const LbView &L, const int x, const int y, const int z, const int pbuf)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    // the patch of this step lives in buffer pbuf (step % 3)
    bool in_patch = (MODE == LAT_NEAR);
    if constexpr (MODE != LAT_NEAR) in_patch = node_in_patch(L, L.ctl, pbuf, x, y, z);
    if (MODE == LAT_FAR && in_patch) return false;
    {
        const int nxy = nx * ny;
        const int node = x + nx * y + nxy * z;
        T *__restrict__ f = static_cast<T *>(L.f);
        // the patch nodes keep their lines in L2 between steps (see L2Keep)
        struct NoKeep {};
        [[maybe_unused]] const std::conditional_t<MODE == LAT_NEAR, P, NoKeep> K;
        const int qs = (int)L.qs;
        const bool px = PER && L.bc[0] == IBL_BC_PERIODIC, py = PER && L.bc[1] == IBL_BC_PERIODIC,
                   pz = PER && L.bc[2] == IBL_BC_PERIODIC;
        const int sx = px ? 0 : (x == 0 ? -1 : (x == nx - 1 ? 1 : 0));
        const int sy = py ? 0 : (y == 0 ? -1 : (y == ny - 1 ? 1 : 0));
        const int sz = pz ? 0 : (z == 0 ? -1 : (z == nz - 1 ? 1 : 0));
        // offsets to the neighbours along each axis (odd step: the sources
        // x - c_i).  Periodic axes wrap.  On a Zou-He axis a missing
        // neighbour points back at the node itself: a population whose source
        // lies outside the box is an unknown that the boundary rebuild below
        // overwrites before anything reads it, so its load only needs an
        // address inside the array, not a guard.  The patch-node update
        // (LAT_NEAR) keeps the guard instead (bits of `miss`: 1 x-1, 2 x+1,
        // 4 y-1, 8 y+1, 16 z-1, 32 z+1), which measured faster there.
        int oxm = -1, oxp = 1, oym = -nx, oyp = nx, ozm = -nxy, ozp = nxy;
        [[maybe_unused]] int miss = 0;
        if constexpr (ODD && MODE == LAT_NEAR) {
            if (x == 0) { if (px) oxm = nx - 1; else miss |= 1; }
            if (x == nx - 1) { if (px) oxp = -(nx - 1); else miss |= 2; }
            if (y == 0) { if (py) oym = (ny - 1) * nx; else miss |= 4; }
            if (y == ny - 1) { if (py) oyp = -(ny - 1) * nx; else miss |= 8; }
            if (z == 0) { if (pz) ozm = (nz - 1) * nxy; else miss |= 16; }
            if (z == nz - 1) { if (pz) ozp = -(nz - 1) * nxy; else miss |= 32; }
        } else if constexpr (ODD) {
            if (x == 0) oxm = px ? nx - 1 : 0;
            if (x == nx - 1) oxp = px ? -(nx - 1) : 0;
            if (y == 0) oym = py ? (ny - 1) * nx : 0;
            if (y == ny - 1) oyp = py ? -(ny - 1) * nx : 0;
            if (z == 0) ozm = pz ? (nz - 1) * nxy : 0;
            if (z == nz - 1) ozp = pz ? -(nz - 1) * nxy : 0;
        }

        T g[19];
        if constexpr (!ODD) {
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                if constexpr (MODE == LAT_NEAR) g[i] = K.ld(f + i * qs + node);
                else g[i] = f[i * qs + node];
            });
        } else {
            // source x - c_i, slot opp(i)
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = cxf(i), cy = cyf(i), cz = czf(i);
                const int off = (cx > 0 ? oxm : (cx < 0 ? oxp : 0)) + (cy > 0 ? oym : (cy < 0 ? oyp : 0)) +
                                (cz > 0 ? ozm : (cz < 0 ? ozp : 0));
                if constexpr (MODE == LAT_NEAR) {
                    constexpr int need = (cx > 0 ? 1 : (cx < 0 ? 2 : 0)) | (cy > 0 ? 4 : (cy < 0 ? 8 : 0)) |
                                         (cz > 0 ? 16 : (cz < 0 ? 32 : 0));
                    g[i] = (miss & need) == 0 ? K.ld(f + opp(i) * qs + node + off) : T(0);
                } else {
                    g[i] = f[opp(i) * qs + node + off];
                }
            });
        }

        return lattice_finish<T, ODD, REC, MODE, PER, P>(L, g, x, y, z, node, in_patch, pbuf, sx, sy, sz);
    }
}

// Closes step t: the step counter becomes t + 1 and the frame of step t + 1
// goes to its parity's slot.  The lattice kernel of step t and the patch
// update of step t read the other slot, and the kernels of step t - 1, the
// last readers of this one, have finished (both are ordered before the
// lattice kernel of step t), so one thread of that kernel can do it while the
// rest of the step runs: no separate launch sits between two lattice updates.
__device__ __forceinline__ void close_step(const LbView &L)
{
    const long long s = L.ctl->step + 1;
    L.ctl->step = s;
    const long long k = s / L.n_hold;
    L.ctl->frame_par[s & 1] = (int)(k < L.n_frames - 1 ? k : L.n_frames - 1);
}

template <typename T, bool ODD, bool REC, int MODE, bool PER>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 8 : 4) k_lattice(LbView L, int pbuf, int ahead)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0) close_step(L);
    // L2 prefetch of this thread's node `ahead` z-planes on, which a block of
    // about one resident wave later updates: its loads then find the lines in
    // L2 instead of waiting on DRAM behind the stream (ahead = 0: none; the
    // host leaves it out for a large droplet patch, see L.prefetch)
    const int za = z + ahead;
    if (ahead > 0 && za < L.n[2] && x < L.n[0] && y < L.n[1]) {
        const T *f = static_cast<const T *>(L.f);
        const int na = x + L.n[0] * (y + L.n[1] * za);
        const int qs = (int)L.qs;
#pragma unroll
        for (int i = 0; i < 19; ++i) asm volatile("prefetch.global.L2 [%0];" ::"l"(f + i * qs + na));
    }
    bool bad = false;
    if (x < L.n[0] && y < L.n[1]) bad = lattice_node<T, ODD, REC, MODE, PER>(L, x, y, z, pbuf);
    // sticky instability flag, one atomic per warp at most
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m != 0u && (threadIdx.x & 31) == 0) atomicOr(&L.ctl->err, IBL_ERRBIT_UNSTABLE);
}

// Outside update (FAR) or whole-box update (FULL) through a shared-memory
// pipeline, for FP32 populations in a box with Zou-He walls on every axis.
// The one-thread-per-node kernel above holds its 19 loads in registers, so
// the bytes it keeps in flight are capped by the resident threads (8 blocks
// of 128 at 64 registers fill the register file), and a droplet-kernel
// block that takes a slot on an SM cuts that SM's share of the stream.
// Here each block is persistent (B per SM) and walks tiles of NT
// consecutive nodes of the flattened box; warp 0 stages the 19 source runs
// of a tile (one lane per run) with bulk asynchronous copies (cp.async.bulk,
// completion counted in bytes on an mbarrier) S tiles ahead, so the bytes in
// flight do not depend on registers.  On GB300 it measures slower than the
// direct kernel in every launch shape (the update is co-limited by
// instruction issue, and the pipeline adds instructions and holds its SM
// resources for the whole launch); it is selected by ibl_set_outside_update.
// Source runs: even step, slot i of the tile's own nodes; odd step, slot
// opp(i) of the nodes n - o_i, o_i = c_ix + c_iy nx + c_iz nx ny (the
// source x - c_i).  A run [n0 - o_i, n0 - o_i + NT) is widened down to the
// 16-byte boundary u_i = (n0 - o_i) & ~3 and up to the next one, and placed
// in its stage slot as if it started at u_i, so that node n0 + t reads
// element t + d_i with d_i = (n0 - o_i) - u_i = (-o_i) & 3 (n0 is a multiple
// of 4), the same for every tile.  The part of a widened run outside its
// array is not copied: those elements, like any other element of a source
// outside the box (a row, plane or array end crossed), are unknowns the
// boundary rebuild overwrites.  Stores go straight from registers
// (lattice_finish).
constexpr unsigned long long kStageWaitNs = 1000000000ull;  // a stage that has not arrived after 1 s is lost
constexpr unsigned long long kDrainWaitNs = 200000000ull;  // then each copy still in flight gets 0.2 s

template <int NT>
__host__ __device__ constexpr int stage_run()
{
    return NT + 8;  // floats per population per stage: NT plus the widening to 16-byte boundaries
}

template <int NT, int S>
__host__ __device__ constexpr size_t stage_bytes()
{
    return sizeof(float) * (size_t)S * 19 * stage_run<NT>();
}

template <bool ODD, int i>
__device__ __forceinline__ int src_offset(const int nx, const int nxy)
{
    return ODD ? cxf(i) + cyf(i) * nx + czf(i) * nxy : 0;
}

// a / b for 0 <= a < 2^26 and b >= 1 from a float reciprocal, corrected to
// the exact quotient
__device__ __forceinline__ int div_by(const int a, const int b, const float inv_b)
{
    int q = __float2int_rz(__int2float_rn(a) * inv_b);
    const int r = a - q * b;
    q += (r >= b) - (r < 0);
    return q;
}

// Registers are capped near 80 per thread whatever the resident blocks B (the
// bound is 6 blocks of 128 threads, or 3 of 256), leaving part of the
// register file free for the droplet kernels beside this one.
template <int NT, int S, int B, bool ODD, int MODE>
__global__ void __launch_bounds__(NT, (B > 768 / NT ? B : 768 / NT)) k_lattice_staged(LbView L, int pbuf)
{
    constexpr int RUN = stage_run<NT>();
    extern __shared__ __align__(128) float stage[];  // [S][19][RUN]
    __shared__ __align__(8) unsigned long long full[S];
    const int tid = threadIdx.x;
    const int nodes = L.nodes, nx = L.n[0], ny = L.n[1], nz = L.n[2], nxy = nx * ny;
    const int qs = (int)L.qs;
    const float *__restrict__ f = static_cast<const float *>(L.f);
    const int ntiles = (nodes + NT - 1) / NT;
    const float inv_nx = 1.0f / (float)nx, inv_nxy = 1.0f / (float)nxy;
    if ((blockIdx.x | tid) == 0) close_step(L);
    if (tid == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&full[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // d_i of every population, two bits each
    unsigned long long dpack = 0;
    if constexpr (ODD)
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            dpack |= (unsigned long long)((-src_offset<ODD, i>(nx, nxy)) & 3) << (2 * i);
        });
    // warp 0: the 19 source runs of `tile` into stage `s`, lane i copying
    // run i.  Lane 0's single arrival, which also announces the bytes of all
    // 19 copies, comes after the copies are issued: until it arrives the
    // phase cannot complete, whatever the copies have delivered by then.
    const int lane = tid & 31;
    int off_l = 0, arr_l = 0;  // lane i < 19: source offset and array of population i
    sfor<19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (lane == i) {
            off_l = src_offset<ODD, i>(nx, nxy);
            arr_l = ODD ? opp(i) : i;
        }
    });
    auto issue = [&](const int tile, const int s) {
        const int n0 = tile * NT, len = min(NT, nodes - n0);
        unsigned nb = 0;
        if (lane < 19) {
            const int u = (n0 - off_l) & ~3;  // widened start, may lie before the array
            const int a = max(u, 0), b = min((n0 - off_l + len + 3) & ~3, qs);
            if (b > a) {
                nb = 4u * (unsigned)(b - a);
                bulk_g2s(stage + (s * 19 + lane) * RUN + (a - u), f + (size_t)arr_l * qs + a, nb, &full[s]);
            }
        }
        const unsigned total = __reduce_add_sync(0xffffffffu, nb);
        // L.stage_fault (tests of the timeout path only): announce 16 bytes
        // more than the copies deliver, so that the phase never completes
        if (lane == 0) mbar_arrive_expect_tx(&full[s], total + (L.stage_fault ? 16u : 0u));
    };
    if (tid < 32)
        for (int k = 0; k < S; ++k) {
            const int t = blockIdx.x + k * gridDim.x;
            if (t < ntiles) issue(t, k);
        }
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int s = k % S;
        const bool arrived = mbar_wait(&full[s], (unsigned)(k / S) & 1u, kStageWaitNs);
        if (!__syncthreads_and(arrived)) {
            // a stage that never completes: report it, let the copies still
            // in flight land (bounded), and leave without touching memory
            if (tid == 0) {
                atomicOr(&L.ctl->err, IBL_ERRBIT_TIMEOUT);
                for (int j = 0; j < S; ++j) {
                    const int kk = k + j;
                    if (blockIdx.x + kk * (int)gridDim.x < ntiles)
                        mbar_wait(&full[kk % S], (unsigned)(kk / S) & 1u, kDrainWaitNs);
                }
            }
            return;
        }
        const int n = tile * NT + tid;
        bool bad = false;
        if (n < nodes) {
            const int z = div_by(n, nxy, inv_nxy), rem = n - z * nxy, y = div_by(rem, nx, inv_nx), x = rem - y * nx;
            const bool in_patch = node_in_patch(L, L.ctl, pbuf, x, y, z);
            if (!(MODE == LAT_FAR && in_patch)) {
                const int sx = x == 0 ? -1 : (x == nx - 1 ? 1 : 0);
                const int sy = y == 0 ? -1 : (y == ny - 1 ? 1 : 0);
                const int sz = z == 0 ? -1 : (z == nz - 1 ? 1 : 0);
                const float *src = stage + s * 19 * RUN + tid;
                float g[19];
                sfor<19>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    if constexpr (ODD) g[i] = src[i * RUN + (int)((dpack >> (2 * i)) & 3u)];
                    else g[i] = src[i * RUN];
                });
                bad = lattice_finish<float, ODD, false, MODE, false>(L, g, x, y, z, n, in_patch, pbuf, sx, sy, sz);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, bad);
        if (m != 0u && (tid & 31) == 0) atomicOr(&L.ctl->err, IBL_ERRBIT_UNSTABLE);
        __syncthreads();  // every thread is done with stage s
        if (tid < 32) {
            const int t = tile + S * (int)gridDim.x;
            if (t < ntiles) issue(t, s);
        }
    }
}

// The patch nodes of the step: one warp per row (y, z) of the patch box,
// its lanes along x (32 at a time), rows grid-strided over the warps of the
// grid, so that each access of a warp is one contiguous run of a row.
template <typename T, bool ODD, bool REC, bool PER, class P>
__device__ __forceinline__ void patch_rows(const LbView &L, const int buf, const int warp0, const int nwarps)
{
    const Ctl *c = L.ctl;
    const int ex = c->patch_ext[buf][0] + 1, ey = c->patch_ext[buf][1] + 1, ez = c->patch_ext[buf][2] + 1;
    const int lx = c->patch_lo[buf][0], ly = c->patch_lo[buf][1], lz = c->patch_lo[buf][2];
    const int rows = (ex > 0 && ey > 0 && ez > 0) ? ey * ez : 0;
    const int lane = threadIdx.x & 31;
    for (int row = warp0; row < rows; row += nwarps) {
        const int pz = row / ey, py = row - pz * ey;
        int y = ly + py, z = lz + pz;
        if (y >= L.n[1]) y -= L.n[1];  // a periodic patch may wrap once
        if (z >= L.n[2]) z -= L.n[2];
        for (int x0 = 0; x0 < ex; x0 += 32) {
            bool bad = false;
            if (x0 + lane < ex) {
                int x = lx + x0 + lane;
                if (x >= L.n[0]) x -= L.n[0];
                bad = lattice_node<T, ODD, REC, LAT_NEAR, PER, P>(L, x, y, z, buf);
            }
            const unsigned m = __ballot_sync(0xffffffffu, bad);
            if (m != 0u && lane == 0) atomicOr(&L.ctl->err, IBL_ERRBIT_UNSTABLE);
        }
    }
}

template <typename T, bool ODD, bool REC, bool PER>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_lattice_near(LbView L, int buf)
{
    const int wpb = blockDim.x >> 5;
    patch_rows<T, ODD, REC, PER, L2Keep>(L, buf, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb);
}

// Ensemble: the nodes outside each member's droplet patch, one launch over
// the lattices of a group of members (the patches are updated concurrently
// by k_lattice_near_batched on the helper stream).  Block b works for member
// blk_member[b0 + b] (view G.v[member - m0], read from the kernel
// parameters) as its local block l = b0 + b - blk_start[member]: NT
// consecutive nodes of z plane l / bpp (bpp = blocks per plane) in x-fastest
// order, starting at node (l mod bpp) NT of the plane; the row of a node is
// p / n_x, taken as floor((p + 1/2) inv_nx), exact while n_x n_y < 2^22 (the
// fraction of (p + 1/2)/n_x stays 1/(2 n_x) away from an integer, more than
// the float rounding).  The first thread of a member's first block closes
// that member's step, as the single-droplet far kernel does.  Each thread
// prefetches into L2 its (x, y) `ahead` planes further (about `waves`
// resident waves of blocks later).
template <typename T, bool ODD, int NT, bool PER>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? 1024 : 512) / NT)
    k_lattice_batched(const __grid_constant__ LbGroup G, const int m0, const int b0,
                      const int *__restrict__ blk_member, const int *__restrict__ blk_start, const int pbuf,
                      const int ahead_nodes)
{
    const int mi = blk_member[b0 + blockIdx.x];
    const LbView &L = G.v[mi - m0];
    const int nx = L.n[0], nxy = L.n[0] * L.n[1];
    const int bpp = (nxy + NT - 1) / NT;
    const int lb = b0 + (int)blockIdx.x - blk_start[mi];
    const int z = lb / bpp;
    const int p = (lb - z * bpp) * NT + (int)threadIdx.x;
    if (lb == 0 && threadIdx.x == 0) close_step(L);
    if (ahead_nodes > 0) {
        const int za = z + (ahead_nodes + nxy - 1) / nxy;
        if (za < L.n[2] && p < nxy) {
            const T *f = static_cast<const T *>(L.f);
            const int na = p + nxy * za;
            const int qs = (int)L.qs;
#pragma unroll
            for (int i = 0; i < 19; ++i) asm volatile("prefetch.global.L2 [%0];" ::"l"(f + i * qs + na));
        }
    }
    bool bad = false;
    if (p < nxy) {
        const int y = (int)(((float)p + 0.5f) * L.inv_nx);
        bad = lattice_node<T, ODD, false, LAT_FAR, PER>(L, p - y * nx, y, z, pbuf);
    }
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m != 0u && (threadIdx.x & 31) == 0) atomicOr(&L.ctl->err, IBL_ERRBIT_UNSTABLE);
}

// Ensemble: the patch nodes of every member of a group (blockIdx.y is the
// member within the group), a warp per patch row as in k_lattice_near.
template <typename T, bool ODD, bool PER, class P>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_lattice_near_batched(const __grid_constant__ LbGroup G,
                                                                                    const int buf)
{
    const int wpb = blockDim.x >> 5;
    patch_rows<T, ODD, false, PER, P>(G.v[blockIdx.y], buf, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb);
}


template <typename T>
__global__ void __launch_bounds__(256) k_init(LbView L)
{
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.nodes) return;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int z = node / (nx * ny);
    const int rem = node - z * nx * ny;
    const int y = rem / nx;
    const int x = rem - y * nx;
    const double *A = L.frames;
    const double lx = x - 0.5 * (nx - 1), ly = y - 0.5 * (ny - 1), lz = z - 0.5 * (nz - 1);
    const double u[3] = {A[0] * lx + A[1] * ly + A[2] * lz, A[3] * lx + A[4] * ly + A[5] * lz,
                         A[6] * lx + A[7] * ly + A[8] * lz};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T *f = static_cast<T *>(L.f);
    sfor<19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const double cu = cxf(i) * u[0] + cyf(i) * u[1] + czf(i) * u[2];
        f[i * L.qs + node] = T(wgt(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
    });
}

// ---------------------------------------------------------------------------
// Immersed boundary.
// Patch of lattice nodes the droplet's stencils can touch, from the node
// bounding box [mn, mx]: floor(mn)-1 .. floor(mx)+2 per axis (periodic axes
// keep the lower corner inside the box and may wrap; Zou-He axes clamp).
// `grow` extra nodes on each side (1 covers the nodes' motion over one more
// step: |u| <= 0.3 keeps floor(r) within one node).
__device__ void write_patch(const LbView &L, const double mn[3], const double mx[3], int buf, int grow)
{
    for (int a = 0; a < 3; ++a) {
        const int n = L.n[a];
        double lo_d = mn[a], hi_d = mx[a];
        if (!(lo_d > -1e8 && lo_d < 1e8) || !(hi_d > -1e8 && hi_d < 1e8) || hi_d < lo_d) {
            L.ctl->patch_lo[buf][a] = 0;
            L.ctl->patch_ext[buf][a] = n - 1;
            continue;
        }
        long long lo = (long long)floor(lo_d) - 1 - grow, hi = (long long)floor(hi_d) + 2 + grow;
        if (L.bc[a] == IBL_BC_PERIODIC) {
            if (hi - lo + 1 >= n) {
                lo = 0;
                hi = n - 1;
            } else {
                long long l2 = lo % n;
                if (l2 < 0) l2 += n;
                hi = l2 + (hi - lo);
                lo = l2;
            }
        } else {
            if (lo < 0) lo = 0;
            if (hi > n - 1) hi = n - 1;
            if (hi < lo) hi = lo;
        }
        L.ctl->patch_lo[buf][a] = (int)lo;
        L.ctl->patch_ext[buf][a] = (int)(hi - lo);
    }
}

// Warp 0 of block 0 of the force/spread kernel of step t: reduce the
// bounding-box rows of r_t left by the previous interpolation (or
// regularisation) into the patch of step t + 1, grown by one node, in
// buffer `buf` (the parity of step t + 1).
template <class P>
__device__ void patch_from_rows(const LbView &L, const MeshView &M, int buf)
{
    const int lane = threadIdx.x & 31;
    const int rows = L.ctl->n_part;
    const P K;
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int k = lane; k < rows; k += 32)
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin(mn[a], K.ld(M.part + 6 * k + a));
            mx[a] = fmax(mx[a], K.ld(M.part + 6 * k + 3 + a));
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fmin(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmax(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if (lane == 0) write_patch(L, mn, mx, buf, 1);
}

// Nodal force F_i = -sigma dA/dx_i (Eq. (pi_drop)) gathered over the
// triangles around node i, then spread with the 4-point delta
// (Eq. (ibm_force_d)(a)) by atomic adds into the Eulerian force.  LANES
// lanes per node: the lanes split the incident triangles (reduced with
// shuffles), then each lane adds 16 / LANES x-rows of four stencil points.
// STORED: m_t comes from M.tm (written by k_tri_moment_batched just before);
// otherwise each lane evaluates it for its triangle (three times per
// triangle in all, but one kernel boundary fewer on the droplet chain of a
// single droplet, which is latency bound).
template <typename T, bool STORED, int LANES, class P = L2Keep>
__device__ __forceinline__ void spread_body(const LbView &L, const MeshView &M, const int blk, const int next_buf)
{
    if (blk == 0 && threadIdx.x < 32) patch_from_rows<P>(L, M, next_buf);
    const int gid = blk * (kIbThreads / LANES) + threadIdx.x / LANES;
    const int lane = threadIdx.x % LANES;
    const bool valid = gid < M.nv;
    const int i = valid ? gid : M.nv - 1;
    const P K;
    double F[3] = {0.0, 0.0, 0.0};
    const int k0 = K.ld(M.n2t_ptr + i), k1 = K.ld(M.n2t_ptr + i + 1);
    for (int k = k0 + lane; k < k1; k += LANES) {
        const int e = K.ld(M.n2t + k);
        const int t = e / 3;
        double m[3];
        if constexpr (STORED) {
            for (int a = 0; a < 3; ++a) m[a] = K.ld(M.tm + 3 * t + a);
        } else {
            tri_moment(M, t, m, K);
        }
        double g[3];
        tri_force_m(M, t, e - 3 * t, m, g, K);
        for (int a = 0; a < 3; ++a) F[a] += g[a];
    }
    for (int o = LANES / 2; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) F[a] += __shfl_xor_sync(0xffffffffu, F[a], o, LANES);
    if (valid && lane == 0) {
        M.fn[3 * i] = F[0];
        M.fn[3 * i + 1] = F[1];
        M.fn[3 * i + 2] = F[2];
        if (M.rec_r) {
            M.rec_r[3 * i] = M.r[3 * i];
            M.rec_r[3 * i + 1] = M.r[3 * i + 1];
            M.rec_r[3 * i + 2] = M.r[3 * i + 2];
        }
    }
    if (M.rec_ctl && blk == 0 && threadIdx.x == 32) {
        // this step's patch buffer; warp 0 writes the next step's
        const int pb = (next_buf + 2) % 3;
        for (int a = 0; a < 4; ++a) {
            M.rec_ctl->patch_lo[pb][a] = L.ctl->patch_lo[pb][a];
            M.rec_ctl->patch_ext[pb][a] = L.ctl->patch_ext[pb][a];
        }
    }
    const NodeStencil S = node_stencil<LANES, P>(L, M.r + 3 * i, lane, &K);
    if (valid && !S.ok && lane == 0) atomicOr(&L.ctl->err, IBL_ERRBIT_WALL);
    if (!valid || !S.ok) return;
    const bool perx = L.bc[0] == IBL_BC_PERIODIC, pery = L.bc[1] == IBL_BC_PERIODIC,
               perz = L.bc[2] == IBL_BC_PERIODIC;
    const int nx = L.n[0], nxy = L.n[0] * L.n[1];
    T *force = static_cast<T *>(L.force);  // [nodes][4]
    const T Fx = T(F[0]), Fy = T(F[1]), Fz = T(F[2]);
    // the lane's (y, z) rows r = lane, lane + LANES, ...: (b, c) = (r & 3, r >> 2)
#pragma unroll
    for (int q = 0; q < 16 / LANES; ++q) {
        const int r = lane + LANES * q, b = r & 3, c = r >> 2;
        T w[4], wy, wz;
        stencil_weights<T>(S, b, c, w, wy, wz);
        const int row =
            wrap_index(S.base[1] + b, L.n[1], pery) * nx + wrap_index(S.base[2] + c, L.n[2], perz) * nxy;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const T dl = w[a] * wy * wz;
            const int id = row + wrap_index(S.base[0] + a, nx, perx);
            K.red_add3(force + 4 * id, Fx * dl, Fy * dl, Fz * dl);
        }
    }
}

// Ensemble: m_t of every triangle of every member at the current positions
// (Eq. (pi_drop)), once per step, for the batched force kernel that follows
// on the same stream; blockIdx.y is the member within the group.
template <class P>
__global__ void __launch_bounds__(128) k_tri_moment_batched(const __grid_constant__ MeshGroup MG)
{
    const MeshView &M = MG.v[blockIdx.y];
    const P K;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M.nt; t += gridDim.x * blockDim.x) {
        double m[3];
        tri_moment(M, t, m, K);
        for (int a = 0; a < 3; ++a) K.st(M.tm + 3 * t + a, m[a]);
    }
}

template <typename T, int LANES>
__global__ void __launch_bounds__(128) k_spread(LbView L, MeshView M, int next_buf, int nblk)
{
    // node groups block-strided: a grid capped below nblk leaves SM slots to
    // the concurrent outside update
    for (int b = blockIdx.x; b < nblk; b += (int)gridDim.x) spread_body<T, false, LANES>(L, M, b, next_buf);
}

// Re-centring (Sec. 3.2: the linearisation is centred on the droplet's
// centre of mass).  kCentreBlocks blocks per droplet sum the volume V and
// first moment m of the region the mesh encloses over the signed tetrahedra
// (box centre, a, b, c) of the triangles, block b taking triangles b, b +
// kCentreBlocks, ... thread by thread.  Each block writes its sums to
// M.cpart; the last block to finish adds the rows in block order
// (deterministic) and stores the step's centre, box centre + m / V, in
// buffer `buf`.  Runs after the interpolation of the previous step and
// before any lattice update of this step.
constexpr int kCentreThreads = 128;

__device__ __forceinline__ void centre_of_mass(const LbView &L, const MeshView &M, const int blk, const int buf)
{
    __shared__ double sh[kCentreThreads / 32][4];
    __shared__ int last;
    const double ref[3] = {0.5 * (L.n[0] - 1), 0.5 * (L.n[1] - 1), 0.5 * (L.n[2] - 1)};
    const L2Keep K;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = blk * kCentreThreads + (int)threadIdx.x; t < M.nt; t += kCentreBlocks * kCentreThreads) {
        double p[3][3];
        for (int c = 0; c < 3; ++c) {
            const int q = K.ld(M.tris + 3 * t + c);
            for (int a = 0; a < 3; ++a) p[c][a] = K.ld(M.r + 3 * q + a) - ref[a];
        }
        double bc[3];
        cross3(p[1], p[2], bc);
        const double vt = (p[0][0] * bc[0] + p[0][1] * bc[1] + p[0][2] * bc[2]) / 6.0;
        v[0] += vt;
        for (int a = 0; a < 3; ++a) v[1 + a] += vt * (p[0][a] + p[1][a] + p[2][a]) / 4.0;
    }
    block_sum<4>(v, sh);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) M.cpart[4 * blk + k] = v[k];
        __threadfence();
        last = atomicAdd(&L.ctl->cen_ticket, 1u) == (unsigned)(kCentreBlocks - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double w[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = 0; b < kCentreBlocks; ++b)
            for (int k = 0; k < 4; ++k) w[k] += __ldcg(M.cpart + 4 * b + k);
        for (int a = 0; a < 3; ++a) L.ctl->centre[buf][a] = ref[a] + w[1 + a] / w[0];
        L.ctl->cen_ticket = 0u;
    }
}

__global__ void __launch_bounds__(kCentreThreads) k_centre(LbView L, MeshView M, int buf)
{
    centre_of_mass(L, M, blockIdx.x, buf);
}

// Viscosity ratio (Sec. 2: droplet viscosity chi mu): the inside flags of the
// patch nodes of step `buf` by the even-odd rule on vertical rays.  One
// thread per triangle (a, b, c): for every lattice column (x, y) of the patch
// whose point q = (x + kRayDx, y + kRayDy) lies strictly inside the
// triangle's xy projection (three edge functions of one sign), the height
// z_c of the triangle over q comes from the barycentric weights, and the
// flags of the patch nodes with z < z_c flip.  A node is inside when an odd
// number of triangles lie above it.  The sub-lattice offsets keep the rays
// off mesh vertices and edges; every operation is a separately rounded IEEE
// one (no contraction), so the flags do not depend on the compiler.  The
// patch covers the droplet, so every inside node is a patch node; the patch
// update reads and clears the flags.
constexpr double kRayDx = 1.4142135623730951e-7, kRayDy = 1.7320508075688772e-7;

__device__ __forceinline__ double edge_fn(double ax, double ay, double bx, double by, double qx, double qy)
{
    return __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(qy, ay)), __dmul_rn(__dsub_rn(by, ay), __dsub_rn(qx, ax)));
}

__global__ void __launch_bounds__(128) k_indicator(LbView L, MeshView M, int buf)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M.nt) return;
    const Ctl *c = L.ctl;
    if (c->patch_ext[buf][0] < 0 || c->patch_ext[buf][1] < 0 || c->patch_ext[buf][2] < 0) return;
    const int lo[3] = {c->patch_lo[buf][0], c->patch_lo[buf][1], c->patch_lo[buf][2]};
    const int hi[3] = {lo[0] + c->patch_ext[buf][0], lo[1] + c->patch_ext[buf][1], lo[2] + c->patch_ext[buf][2]};
    double p[3][3];
    for (int k = 0; k < 3; ++k) {
        const int v = M.tris[3 * t + k];
        for (int a = 0; a < 3; ++a) p[k][a] = M.r[3 * v + a];
    }
    const double xmin = fmin(p[0][0], fmin(p[1][0], p[2][0])), xmax = fmax(p[0][0], fmax(p[1][0], p[2][0]));
    const double ymin = fmin(p[0][1], fmin(p[1][1], p[2][1])), ymax = fmax(p[0][1], fmax(p[1][1], p[2][1]));
    int x0 = (int)ceil(__dsub_rn(xmin, kRayDx)), x1 = (int)floor(__dsub_rn(xmax, kRayDx));
    int y0 = (int)ceil(__dsub_rn(ymin, kRayDy)), y1 = (int)floor(__dsub_rn(ymax, kRayDy));
    x0 = max(x0, max(lo[0], 0));
    y0 = max(y0, max(lo[1], 0));
    x1 = min(x1, min(hi[0], L.n[0] - 1));
    y1 = min(y1, min(hi[1], L.n[1] - 1));
    const int z_lo = max(lo[2], 0), z_hi = min(hi[2], L.n[2] - 1);
    for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
            const double qx = __dadd_rn((double)x, kRayDx), qy = __dadd_rn((double)y, kRayDy);
            const double e0 = edge_fn(p[0][0], p[0][1], p[1][0], p[1][1], qx, qy);
            const double e1 = edge_fn(p[1][0], p[1][1], p[2][0], p[2][1], qx, qy);
            const double e2 = edge_fn(p[2][0], p[2][1], p[0][0], p[0][1], qx, qy);
            const bool inside = (e0 > 0.0 && e1 > 0.0 && e2 > 0.0) || (e0 < 0.0 && e1 < 0.0 && e2 < 0.0);
            if (!inside) continue;
            const double num = __dadd_rn(__dadd_rn(__dmul_rn(e1, p[0][2]), __dmul_rn(e2, p[1][2])), __dmul_rn(e0, p[2][2]));
            const double zc = __ddiv_rn(num, __dadd_rn(__dadd_rn(e0, e1), e2));
            for (int z = z_lo; z <= z_hi && (double)z < zc; ++z) {
                const int node = x + L.n[0] * (y + L.n[1] * z);
                atomicXor(L.ind + (node >> 2), 1u << (8 * (node & 3)));
            }
        }
}

// Ensemble version: blockIdx.y is the member within the group.
__global__ void __launch_bounds__(kCentreThreads)
    k_centre_batched(const __grid_constant__ LbGroup LG, const __grid_constant__ MeshGroup MG, int buf)
{
    centre_of_mass(LG.v[blockIdx.y], MG.v[blockIdx.y], blockIdx.x, buf);
}

template <typename T, int LANES, class P = L2Keep>
__device__ __forceinline__ void interp_body(const LbView &L, const MeshView &M, const int blk, const int nblk)
{
    const int gid = blk * (kIbThreads / LANES) + threadIdx.x / LANES;
    const int lane = threadIdx.x % LANES;
    const bool valid = gid < M.nv;
    const int i = valid ? gid : M.nv - 1;
    const P K;
    const NodeStencil S = node_stencil<LANES, P>(L, M.r + 3 * i, lane, &K);
    T v[3] = {T(0), T(0), T(0)};
    if (S.ok) {
        const bool perx = L.bc[0] == IBL_BC_PERIODIC, pery = L.bc[1] == IBL_BC_PERIODIC,
                   perz = L.bc[2] == IBL_BC_PERIODIC;
        const int nx = L.n[0], nxy = L.n[0] * L.n[1];
        const T *vel = static_cast<const T *>(L.vel);  // [nodes][4]
        // the lane's (y, z) rows r = lane, lane + LANES, ...: (b, c) = (r & 3, r >> 2)
#pragma unroll
        for (int q = 0; q < 16 / LANES; ++q) {
            const int r = lane + LANES * q, b = r & 3, c = r >> 2;
            T w[4], wy, wz;
            stencil_weights<T>(S, b, c, w, wy, wz);
            const int row =
                wrap_index(S.base[1] + b, L.n[1], pery) * nx + wrap_index(S.base[2] + c, L.n[2], perz) * nxy;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const T dl = w[a] * wy * wz;
                const int id = row + wrap_index(S.base[0] + a, nx, perx);
                T ua, ub, uc;
                K.ld3(vel + 4 * id, ua, ub, uc);
                v[0] += ua * dl;
                v[1] += ub * dl;
                v[2] += uc * dl;
            }
        }
    }
    for (int o = LANES / 2; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o, LANES);
    const bool have = valid && lane == 0;
    double r[3] = {0.0, 0.0, 0.0};
    if (have) {
        r[0] = K.ld(M.r + 3 * i);
        r[1] = K.ld(M.r + 3 * i + 1);
        r[2] = K.ld(M.r + 3 * i + 2);
        if (!S.ok) {
            atomicOr(&L.ctl->err, IBL_ERRBIT_WALL);
        } else {
            r[0] += (double)v[0];
            r[1] += (double)v[1];
            r[2] += (double)v[2];
            K.st(M.r + 3 * i, r[0]);
            K.st(M.r + 3 * i + 1, r[1]);
            K.st(M.r + 3 * i + 2, r[2]);
        }
    }
    // block min / max of the new positions -> one partial row per block; the
    // next force/spread kernel reduces the rows into the patch (no tail here)
    __shared__ double smn[3][4], smx[3][4];
    const int wlane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = 0; a < 3; ++a) {
        // lanes 0, LANES, 2 LANES, ... hold the warp's nodes
        double mn = have ? r[a] : 1e300, mx = have ? r[a] : -1e300;
        for (int o = LANES; o < 32; o <<= 1) {
            mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (wlane == 0) {
            smn[a][warp] = mn;
            smx[a][warp] = mx;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            double mn = smn[a][0], mx = smx[a][0];
            for (int w = 1; w < nw; ++w) {
                mn = fmin(mn, smn[a][w]);
                mx = fmax(mx, smx[a][w]);
            }
            K.st(M.part + 6 * blk + a, mn);
            K.st(M.part + 6 * blk + 3 + a, mx);
        }
        if (blk == 0) L.ctl->n_part = nblk;
    }
}

template <typename T, int LANES>
__global__ void __launch_bounds__(128) k_interp(LbView L, MeshView M, int nblk)
{
    for (int b = blockIdx.x; b < nblk; b += (int)gridDim.x) {
        interp_body<T, LANES>(L, M, b, nblk);
        __syncthreads();  // the next pass reuses the body's shared rows
    }
}

// Ensemble versions: block b works for member blk_member[b0 + b] as its
// local block b0 + b - blk_start[member]; node-group kernels use ceil(nv/8)
// blocks per member.

// The node groups b0 .. b0 + nb - 1 of a group of members, block-strided so
// that a grid capped below nb leaves most SM slots to the concurrent
// lattice update.
template <typename T, class P>
__global__ void __launch_bounds__(128)
    k_spread_batched(const __grid_constant__ LbGroup LG, const __grid_constant__ MeshGroup MG, const int m0,
                     const int b0, const int nb, const int *__restrict__ blk_member,
                     const int *__restrict__ blk_start, const int next_buf)
{
    for (int bb = b0 + (int)blockIdx.x; bb < b0 + nb; bb += (int)gridDim.x) {
        const int mi = blk_member[bb];
        spread_body<T, true, kFwdLanes, P>(LG.v[mi - m0], MG.v[mi - m0], bb - blk_start[mi], next_buf);
    }
}

template <typename T, class P>
__global__ void __launch_bounds__(128)
    k_interp_batched(const __grid_constant__ LbGroup LG, const __grid_constant__ MeshGroup MG, const int m0,
                     const int b0, const int nb, const int *__restrict__ blk_member,
                     const int *__restrict__ blk_start)
{
    for (int bb = b0 + (int)blockIdx.x; bb < b0 + nb; bb += (int)gridDim.x) {
        const int mi = blk_member[bb];
        interp_body<T, kFwdLanes, P>(LG.v[mi - m0], MG.v[mi - m0], bb - blk_start[mi],
                                     blk_start[mi + 1] - blk_start[mi]);
        __syncthreads();  // the next pass reuses the body's shared rows
    }
}

__device__ void block_bbox_patch(const LbView &L, const MeshView &M, const double *r, int nv, int buf)
{
    __shared__ double sh[32];
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        double lo = 1e300, hi = -1e300;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            lo = fmin(lo, r[3 * i + a]);
            hi = fmax(hi, r[3 * i + a]);
        }
        mn[a] = -block_max(-lo, sh);
        mx[a] = block_max(hi, sh);
    }
    if (threadIdx.x == 0) {
        write_patch(L, mn, mx, buf, 1);
        for (int a = 0; a < 3; ++a) {
            M.part[a] = mn[a];
            M.part[3 + a] = mx[a];
        }
        L.ctl->n_part = 1;
    }
}

// Mesh regularisation, Sec. 3.3, one block: x_o fixed, x_q the previous
// iterate, x_p the new one (ping-pong between r and s1), x_b in s2.
// patch_buf: patch buffer (parity) of the next step, rewritten from the
// regularised positions.
// This thread's share of the enclosed volume and of its first moment, summed
// over signed tetrahedra (x_0, a, b, c) of the triangles, positions relative
// to node 0: v[0] = V, v[1..3] = int (x - x_0) dV.
__device__ __forceinline__ void enclosed_volume_sums(const MeshView &M, double v[4])
{
    v[0] = v[1] = v[2] = v[3] = 0.0;
    const double r0[3] = {M.r[0], M.r[1], M.r[2]};
    for (int t = threadIdx.x; t < M.nt; t += blockDim.x) {
        double pp[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) pp[k][a] = M.r[3 * M.tris[3 * t + k] + a] - r0[a];
        double bc[3];
        cross3(pp[1], pp[2], bc);
        const double vt = (pp[0][0] * bc[0] + pp[0][1] * bc[1] + pp[0][2] * bc[2]) / 6.0;
        v[0] += vt;
        for (int a = 0; a < 3; ++a) v[1 + a] += vt * (pp[0][a] + pp[1][a] + pp[2][a]) / 4.0;
    }
}

__global__ void __launch_bounds__(1024) k_regularize(LbView L, MeshView M, RegParams p, int patch_buf)
{
    __shared__ double sh[32];
    const int nv = M.nv;
    // mesh quality: the largest ratio of longest to shortest edge over the
    // triangles (node clustering and loose, stretched elements both raise it)
    double q = 1.0;
    for (int t = threadIdx.x; t < M.nt; t += blockDim.x) {
        const int v[3] = {M.tris[3 * t], M.tris[3 * t + 1], M.tris[3 * t + 2]};
        double e2[3];
        for (int k = 0; k < 3; ++k) {
            const double *a = M.r + 3 * v[k], *b = M.r + 3 * v[(k + 1) % 3];
            const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
            e2[k] = dx * dx + dy * dy + dz * dz;
        }
        const double lo = fmin(e2[0], fmin(e2[1], e2[2])), hi = fmax(e2[0], fmax(e2[1], e2[2]));
        q = fmax(q, lo > 0.0 ? sqrt(hi / lo) : 1e300);
    }
    q = block_max(q, sh);
    if (threadIdx.x == 0) L.ctl->mesh_q = q;
    if (p.trigger > 0.0 && !(q > p.trigger)) {
        // adaptive schedule: the mesh is still regular enough, nothing to do
        if (threadIdx.x == 0) L.ctl->reg_iters = 0;
        return;
    }
    __shared__ double shv[32][4];
    double V0 = 0.0;
    if (p.keep_volume) {
        double v4[4];
        enclosed_volume_sums(M, v4);
        block_sum<4>(v4, shv);
        V0 = v4[0];
    }
    double *xo = M.s0, *xb = M.s2;
    double *buf[2] = {M.r, M.s1};
    for (int i = threadIdx.x; i < 3 * nv; i += blockDim.x) xo[i] = M.r[i];
    __syncthreads();
    const double sg = p.plus_sign ? 1.0 : -1.0;
    int cur = 0, it = 0;
    bool conv = false;
    while (it < p.max_iter) {
        ++it;
        const double *xq = buf[cur];
        double *xp = buf[cur ^ 1];
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            const int b0 = M.nb_ptr[i], b1 = M.nb_ptr[i + 1];
            const int ni = b1 - b0;
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = b0; k < b1; ++k) s += xq[3 * M.nb_idx[k] + a];
                const double v = p.alpha * xo[3 * i + a] + (1.0 - p.alpha) / ni * s;
                xp[3 * i + a] = v;
                xb[3 * i + a] = v - (p.alpha * xo[3 * i + a] + (1.0 - p.alpha) * xq[3 * i + a]);
            }
        }
        __syncthreads();
        double dmax = 0.0;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            const int b0 = M.nb_ptr[i], b1 = M.nb_ptr[i + 1];
            const int ni = b1 - b0;
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = b0; k < b1; ++k) s += xb[3 * M.nb_idx[k] + a];
                const double v = xp[3 * i + a] - (p.gamma * xb[3 * i + a] + sg * (1.0 - p.gamma) / ni * s);
                xp[3 * i + a] = v;
                const double d = v - xq[3 * i + a];
                d2 += d * d;
            }
            dmax = fmax(dmax, sqrt(d2));
        }
        dmax = block_max(dmax, sh);  // includes a barrier after the writes above
        cur ^= 1;
        if (dmax < p.tol) {
            conv = true;
            break;
        }
    }
    if (cur != 0) {
        for (int i = threadIdx.x; i < 3 * nv; i += blockDim.x) M.r[i] = M.s1[i];
    }
    __syncthreads();
    if (p.keep_volume) {
        // scale about the volume centroid back to the volume enclosed before
        double v4[4];
        enclosed_volume_sums(M, v4);
        block_sum<4>(v4, shv);
        const double c[3] = {M.r[0] + v4[1] / v4[0], M.r[1] + v4[2] / v4[0], M.r[2] + v4[3] / v4[0]};
        const double f = cbrt(V0 / v4[0]);
        __syncthreads();  // every thread has read M.r[0..2] before it moves
        for (int i = threadIdx.x; i < nv; i += blockDim.x)
            for (int a = 0; a < 3; ++a) M.r[3 * i + a] = c[a] + f * (M.r[3 * i + a] - c[a]);
        __syncthreads();
    }
    block_bbox_patch(L, M, M.r, nv, patch_buf);
    if (threadIdx.x == 0) {
        L.ctl->reg_iters = it;
        L.ctl->reg_count += 1;
        if (!conv) atomicOr(&L.ctl->err, IBL_ERRBIT_NOCONV);
    }
}

// The same regularisation on a thread-block cluster of kRegCluster CTAs
// (one per SM), for meshes of up to kRegCluster * kRegPerCta nodes.  CTA c
// owns nodes [c P, c P + P) and keeps their original position, the two
// iterates and the correction b in its shared memory; neighbours owned by
// other CTAs are read through distributed shared memory.  The hardware
// cluster barrier separates the phases, and each CTA reduces the maxima and
// sums published by all CTAs in the same order, so every CTA takes the same
// decisions.  The per-triangle passes (quality, volumes) and the node
// updates spread over the cluster's SMs instead of one.
namespace cg = cooperative_groups;
constexpr int kRegCluster = 16;
constexpr int kRegPerCta = 2048;

__global__ void __launch_bounds__(1024) k_regularize_cluster(LbView L, MeshView M, RegParams p, int patch_buf, int P)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int nv = M.nv, tid = threadIdx.x, nth = blockDim.x;
    extern __shared__ double sm[];
    double *xo = sm, *xa = sm + 3 * P, *xc = sm + 6 * P, *xb = sm + 9 * P;
    double *red = sm + 12 * P;  // [8] values this CTA publishes to the cluster
    __shared__ double shr[32];
    __shared__ double sh4[32][4];
    const int g0 = rank * P, g1 = min(nv, g0 + P), own = max(0, g1 - g0);
    // cluster-wide max / sum of values published in red[0..k) by every CTA
    auto cluster_max = [&](double v) -> double {
        v = block_max(v, shr);
        if (tid == 0) red[0] = v;
        cluster.sync();
        double m = -1e300;
        for (int c = 0; c < C; ++c) m = fmax(m, *cluster.map_shared_rank(red, c));
        cluster.sync();  // the slot is reused by the next reduction
        return m;
    };
    auto cluster_sum4 = [&](double (&v)[4]) {
        block_sum<4>(v, sh4);
        if (tid < 4) red[tid] = v[tid];
        cluster.sync();
        for (int k = 0; k < 4; ++k) {
            double s = 0.0;
            for (int c = 0; c < C; ++c) s += cluster.map_shared_rank(red, c)[k];
            v[k] = s;
        }
        cluster.sync();
    };
    // position of node j in the iterate `buf` (xa or xc), wherever it lives
    auto pos = [&](double *buf, int j, int a) -> double {
        const int c = j / P;
        return cluster.map_shared_rank(buf, c)[3 * (j - c * P) + a];
    };
    // mesh quality over the triangles, from the positions in global memory
    double q = 1.0;
    for (int t = rank * nth + tid; t < M.nt; t += C * nth) {
        const int v[3] = {M.tris[3 * t], M.tris[3 * t + 1], M.tris[3 * t + 2]};
        double e2[3];
        for (int k = 0; k < 3; ++k) {
            const double *a = M.r + 3 * v[k], *b = M.r + 3 * v[(k + 1) % 3];
            const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
            e2[k] = dx * dx + dy * dy + dz * dz;
        }
        const double lo = fmin(e2[0], fmin(e2[1], e2[2])), hi = fmax(e2[0], fmax(e2[1], e2[2]));
        q = fmax(q, lo > 0.0 ? sqrt(hi / lo) : 1e300);
    }
    q = cluster_max(q);
    if (rank == 0 && tid == 0) L.ctl->mesh_q = q;
    if (p.trigger > 0.0 && !(q > p.trigger)) {
        if (rank == 0 && tid == 0) L.ctl->reg_iters = 0;
        return;
    }
    const double r0[3] = {M.r[0], M.r[1], M.r[2]};
    double V0 = 0.0;
    if (p.keep_volume) {
        double v4[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = rank * nth + tid; t < M.nt; t += C * nth) {
            double pp[3][3];
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 3; ++a) pp[k][a] = M.r[3 * M.tris[3 * t + k] + a] - r0[a];
            double bc[3];
            cross3(pp[1], pp[2], bc);
            v4[0] += (pp[0][0] * bc[0] + pp[0][1] * bc[1] + pp[0][2] * bc[2]) / 6.0;
        }
        cluster_sum4(v4);
        V0 = v4[0];
    }
    for (int l = tid; l < own; l += nth)
        for (int a = 0; a < 3; ++a) xo[3 * l + a] = xa[3 * l + a] = M.r[3 * (g0 + l) + a];
    cluster.sync();
    const double sg = p.plus_sign ? 1.0 : -1.0;
    double *xq = xa, *xp = xc;
    int it = 0;
    bool conv = false;
    while (it < p.max_iter) {
        ++it;
        // Eq. (extended laplacian smoothing) and Eq. (distanceregularization)
        for (int l = tid; l < own; l += nth) {
            const int g = g0 + l, b0 = M.nb_ptr[g], b1 = M.nb_ptr[g + 1], ni = b1 - b0;
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = b0; k < b1; ++k) s += pos(xq, M.nb_idx[k], a);
                const double v = p.alpha * xo[3 * l + a] + (1.0 - p.alpha) / ni * s;
                xp[3 * l + a] = v;
                xb[3 * l + a] = v - (p.alpha * xo[3 * l + a] + (1.0 - p.alpha) * xq[3 * l + a]);
            }
        }
        cluster.sync();
        // Eq. (HC_algo_full) and the exit test
        double dmax = 0.0;
        for (int l = tid; l < own; l += nth) {
            const int g = g0 + l, b0 = M.nb_ptr[g], b1 = M.nb_ptr[g + 1], ni = b1 - b0;
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = b0; k < b1; ++k) s += pos(xb, M.nb_idx[k], a);
                const double v = xp[3 * l + a] - (p.gamma * xb[3 * l + a] + sg * (1.0 - p.gamma) / ni * s);
                xp[3 * l + a] = v;
                const double d = v - xq[3 * l + a];
                d2 += d * d;
            }
            dmax = fmax(dmax, sqrt(d2));
        }
        dmax = cluster_max(dmax);  // its barriers also end every read of xb and xq
        double *tmp = xq;
        xq = xp;
        xp = tmp;
        if (dmax < p.tol) {
            conv = true;
            break;
        }
    }
    // xq holds the result
    double c[3] = {0.0, 0.0, 0.0}, f = 1.0;
    if (p.keep_volume) {
        double v4[4] = {0.0, 0.0, 0.0, 0.0};
        const double s0[3] = {pos(xq, 0, 0), pos(xq, 0, 1), pos(xq, 0, 2)};
        for (int t = rank * nth + tid; t < M.nt; t += C * nth) {
            double pp[3][3];
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 3; ++a) pp[k][a] = pos(xq, M.tris[3 * t + k], a) - s0[a];
            double bc[3];
            cross3(pp[1], pp[2], bc);
            const double vt = (pp[0][0] * bc[0] + pp[0][1] * bc[1] + pp[0][2] * bc[2]) / 6.0;
            v4[0] += vt;
            for (int a = 0; a < 3; ++a) v4[1 + a] += vt * (pp[0][a] + pp[1][a] + pp[2][a]) / 4.0;
        }
        cluster_sum4(v4);
        for (int a = 0; a < 3; ++a) c[a] = s0[a] + v4[1 + a] / v4[0];
        f = cbrt(V0 / v4[0]);
    }
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int l = tid; l < own; l += nth)
        for (int a = 0; a < 3; ++a) {
            const double v = p.keep_volume ? c[a] + f * (xq[3 * l + a] - c[a]) : xq[3 * l + a];
            M.r[3 * (g0 + l) + a] = v;
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    for (int a = 0; a < 3; ++a) {
        mn[a] = -cluster_max(-mn[a]);
        mx[a] = cluster_max(mx[a]);
    }
    if (rank == 0 && tid == 0) {
        write_patch(L, mn, mx, patch_buf, 1);
        for (int a = 0; a < 3; ++a) {
            M.part[a] = mn[a];
            M.part[3 + a] = mx[a];
        }
        L.ctl->n_part = 1;
        L.ctl->reg_iters = it;
        L.ctl->reg_count += 1;
        if (!conv) atomicOr(&L.ctl->err, IBL_ERRBIT_NOCONV);
    }
}

__global__ void __launch_bounds__(256) k_patch(LbView L, MeshView M, int buf)
{
    block_bbox_patch(L, M, M.r, M.nv, buf);
}

// Shape record (Sec. 2): enclosed volume, centroid and second moment by
// signed tetrahedra (ref, a, b, c), S = (5/V) M, eigen-decomposition, Taylor
// D and beta of Eq. (beta).  Block blk of nblk sums its share of the
// triangles; the last block to finish (a ticket in the control block) adds
// the partial sums in block order and writes the record.
__device__ __forceinline__ void observables_body(const LbView &L, const MeshView &M, const unsigned blk,
                                                 const unsigned nblk)
{
    __shared__ double sh11[8][11];
    __shared__ bool last;
    // volume integrals relative to node 0 (any point near the droplet will
    // do; this one needs no prior reduction)
    const double ref[3] = {M.r[0], M.r[1], M.r[2]};
    double acc[11];
    for (int k = 0; k < 11; ++k) acc[k] = 0.0;
    for (int t = blk * blockDim.x + threadIdx.x; t < M.nt; t += nblk * blockDim.x) {
        double p[3][3];
        for (int v = 0; v < 3; ++v) {
            const int id = M.tris[3 * t + v];
            for (int a = 0; a < 3; ++a) p[v][a] = M.r[3 * id + a] - ref[a];
        }
        double bc[3];
        cross3(p[1], p[2], bc);
        const double vt = (p[0][0] * bc[0] + p[0][1] * bc[1] + p[0][2] * bc[2]) / 6.0;
        const double s[3] = {p[0][0] + p[1][0] + p[2][0], p[0][1] + p[1][1] + p[2][1],
                             p[0][2] + p[1][2] + p[2][2]};
        acc[0] += vt;
        for (int a = 0; a < 3; ++a) acc[1 + a] += vt * s[a];
        // second moments xx, yy, zz, xy, xz, yz of a, b, c and s
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
        double e1[3], e2[3], nn[3];
        for (int a = 0; a < 3; ++a) { e1[a] = p[1][a] - p[0][a]; e2[a] = p[2][a] - p[0][a]; }
        cross3(e1, e2, nn);
        acc[10] += 0.5 * sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    }
    // per-block partial sums; the last block adds them in block order
    block_sum<11>(acc, sh11);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 11; ++k) M.obs_part[11 * blk + k] = acc[k];
        __threadfence();
        const unsigned t = atomicAdd(&L.ctl->obs_blocks_done, 1u);
        last = (t == nblk - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    for (int k = 0; k < 11; ++k) acc[k] = 0.0;
    for (unsigned b = 0; b < nblk; ++b)
        for (int k = 0; k < 11; ++k) acc[k] += __ldcg(M.obs_part + 11 * b + k);
    L.ctl->obs_blocks_done = 0u;
    const double V = acc[0];
    double xc[3];
    for (int a = 0; a < 3; ++a) xc[a] = acc[1 + a] / 4.0 / V;
    double S6[6];
    for (int k = 0; k < 6; ++k) S6[k] = acc[4 + k] / 20.0;
    S6[0] -= V * xc[0] * xc[0];
    S6[1] -= V * xc[1] * xc[1];
    S6[2] -= V * xc[2] * xc[2];
    S6[3] -= V * xc[0] * xc[1];
    S6[4] -= V * xc[0] * xc[2];
    S6[5] -= V * xc[1] * xc[2];
    for (int k = 0; k < 6; ++k) S6[k] *= 5.0 / V;
    double a[3][3] = {{S6[0], S6[3], S6[4]}, {S6[3], S6[1], S6[5]}, {S6[4], S6[5], S6[2]}};
    double lam[3], vec[3][3];
    jacobi3(a, lam, vec);
    int order[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[order[j]] < lam[order[i]]) {
                const int t = order[i];
                order[i] = order[j];
                order[j] = t;
            }
    ibl_observables o;
    const long long step = L.ctl->step;
    const long long used = step > 0 ? step - 1 : 0;
    long long kf = used / L.n_hold;
    if (kf > L.n_frames - 1) kf = L.n_frames - 1;
    const double *A = L.frames + 9 * kf;
    o.step = step;
    o.frame = (int)kf;
    o.reg_iters = L.ctl->reg_iters;
    o.err = L.ctl->err;
    o.pad_ = 0;
    o.volume = V;
    o.area = acc[10];
    for (int k = 0; k < 3; ++k) o.centroid[k] = xc[k] + ref[k];
    for (int k = 0; k < 6; ++k) o.S[k] = S6[k];
    for (int k = 0; k < 3; ++k) o.lam[k] = lam[order[k]];
    for (int k = 0; k < 3; ++k) o.vmax[k] = vec[k][order[2]];
    const double sl = sqrt(fmax(o.lam[2], 0.0)), ss = sqrt(fmax(o.lam[0], 0.0));
    o.D = (sl - ss) / (sl + ss);
    double E[3][3], nE = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            E[r][c] = 0.5 * (A[3 * r + c] + A[3 * c + r]);
            nE += E[r][c] * E[r][c];
        }
    nE = sqrt(nE);
    double vEv = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) vEv += o.vmax[r] * E[r][c] * o.vmax[c];
    o.beta = nE > 0.0 ? vEv / nE : __longlong_as_double(0x7ff8000000000000ll);
    const int slot = L.ctl->n_records % M.ring_cap;
    M.ring[slot] = o;
    L.ctl->n_records += 1;
}

__global__ void __launch_bounds__(256) k_observables(LbView L, MeshView M)
{
    observables_body(L, M, blockIdx.x, gridDim.x);
}

// Ensemble: the shape records of the members of a group whose bit is set in
// `due` (blockIdx.y is the member within the group), all in one launch.
__global__ void __launch_bounds__(256) k_observables_batched(const __grid_constant__ LbGroup LG,
                                                             const __grid_constant__ MeshGroup MG,
                                                             const unsigned long long due)
{
    if (!((due >> blockIdx.y) & 1ull)) return;
    observables_body(LG.v[blockIdx.y], MG.v[blockIdx.y], blockIdx.x, gridDim.x);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
static inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// Multiprocessors of the current device (read once; launch shapes and
// prefetch distances are sized by it).
static int sm_count()
{
    static int sms = 0;
    if (sms == 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) sms = 1;
    return sms;
}

cudaError_t launch_init(const LbView &L, cudaStream_t s)
{
    const unsigned g = blocks_for(L.nodes, 256);
    if (L.precision == IBL_FP64) k_init<double><<<g, 256, 0, s>>>(L);
    else k_init<float><<<g, 256, 0, s>>>(L);
    return cudaGetLastError();
}

static void lattice_grid(const LbView &L, dim3 &grid, dim3 &block)
{
    // 128-thread blocks (8 per SM at 64 registers): a concurrently running
    // droplet-kernel block then displaces an eighth of an SM's lattice work
    // rather than a quarter
    const int bx = L.n[0] >= 128 ? 128 : ((L.n[0] + 31) / 32) * 32;
    const int by = 128 / bx;
    block = dim3(bx, by, 1);
    grid = dim3((L.n[0] + bx - 1) / bx, (L.n[1] + by - 1) / by, L.n[2]);
}

static bool any_periodic(const LbView &L)
{
    return L.bc[0] == IBL_BC_PERIODIC || L.bc[1] == IBL_BC_PERIODIC || L.bc[2] == IBL_BC_PERIODIC;
}

template <typename T, bool ODD, bool REC>
static void lattice_launch_t(const LbView &L, int mode, int pbuf, dim3 g, dim3 b, cudaStream_t s)
{
    // prefetch distance: the z-planes one wave of resident blocks covers
    const long long wave = (long long)sm_count() * (sizeof(T) == 4 ? 8 : 4), plane = (long long)g.x * g.y;
    const int ahead = L.prefetch ? (int)((wave + plane - 1) / plane) : 0;
    if (any_periodic(L)) {
        if (mode == LAT_FAR) k_lattice<T, ODD, REC, LAT_FAR, true><<<g, b, 0, s>>>(L, pbuf, ahead);
        else k_lattice<T, ODD, REC, LAT_FULL, true><<<g, b, 0, s>>>(L, pbuf, ahead);
    } else {
        if (mode == LAT_FAR) k_lattice<T, ODD, REC, LAT_FAR, false><<<g, b, 0, s>>>(L, pbuf, ahead);
        else k_lattice<T, ODD, REC, LAT_FULL, false><<<g, b, 0, s>>>(L, pbuf, ahead);
    }
}

// Opts a kernel into its dynamic shared memory and the largest shared-memory
// carveout, once per kernel and device.
static cudaError_t prefer_shared(const void *kernel, size_t dyn)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) done.insert({kernel, dev});
    return e;
}

// Launch shapes of the staged outside update: nodes per tile (= threads per
// block), pipeline stages, resident blocks per SM.
template <int V>
struct StagedShape;
template <>
struct StagedShape<1> {
    static constexpr int NT = 128, S = 2, B = 8;
};
template <>
struct StagedShape<2> {
    static constexpr int NT = 128, S = 3, B = 6;
};

template <int V, bool ODD>
static cudaError_t staged_launch(const LbView &L, int mode, int pbuf, cudaStream_t s)
{
    constexpr int NT = StagedShape<V>::NT, S = StagedShape<V>::S, B = StagedShape<V>::B;
    constexpr size_t smem = stage_bytes<NT, S>();
    void (*k)(LbView, int) = mode == LAT_FAR ? k_lattice_staged<NT, S, B, ODD, LAT_FAR>
                                             : k_lattice_staged<NT, S, B, ODD, LAT_FULL>;
    cudaError_t e = prefer_shared(reinterpret_cast<const void *>(k), smem);
    if (e != cudaSuccess) return e;
    const long long tiles = ((long long)L.nodes + NT - 1) / NT;
    const unsigned g = (unsigned)std::min<long long>(tiles, (long long)sm_count() * B);
    k<<<g, NT, smem, s>>>(L, pbuf);
    return cudaGetLastError();
}

template <bool ODD>
static cudaError_t staged_dispatch(const LbView &L, int mode, int pbuf, cudaStream_t s)
{
    switch (L.staged) {
    case 1: return staged_launch<1, ODD>(L, mode, pbuf, s);
    default: return staged_launch<2, ODD>(L, mode, pbuf, s);
    }
}

template <int V>
static cudaError_t staged_prepare_v()
{
    constexpr int NT = StagedShape<V>::NT, S = StagedShape<V>::S, B = StagedShape<V>::B;
    constexpr size_t smem = stage_bytes<NT, S>();
    cudaError_t e = cudaSuccess;
    for (void (*k)(LbView, int) : {k_lattice_staged<NT, S, B, false, LAT_FAR>, k_lattice_staged<NT, S, B, false, LAT_FULL>,
                                   k_lattice_staged<NT, S, B, true, LAT_FAR>, k_lattice_staged<NT, S, B, true, LAT_FULL>})
        if (e == cudaSuccess) e = prefer_shared(reinterpret_cast<const void *>(k), smem);
    return e;
}

cudaError_t staged_prepare(int kind)
{
    switch (kind) {
    case 1: return staged_prepare_v<1>();
    case 2: return staged_prepare_v<2>();
    default: return cudaSuccess;
    }
}

bool staged_ok(const LbView &L)
{
    return L.precision == IBL_FP32_DEV && !any_periodic(L) && (reinterpret_cast<uintptr_t>(L.f) & 15u) == 0 &&
           (L.qs & 3) == 0 && L.nodes < (1 << 26);
}

cudaError_t launch_lattice(const LbView &L, bool odd, bool record, int mode, int pbuf, cudaStream_t s)
{
    if (L.staged > 0 && !record && staged_ok(L))
        return odd ? staged_dispatch<true>(L, mode, pbuf, s) : staged_dispatch<false>(L, mode, pbuf, s);
    dim3 g, b;
    lattice_grid(L, g, b);
    if (L.precision == IBL_FP64) {
        if (odd) {
            if (record) lattice_launch_t<double, true, true>(L, mode, pbuf, g, b, s);
            else lattice_launch_t<double, true, false>(L, mode, pbuf, g, b, s);
        } else {
            if (record) lattice_launch_t<double, false, true>(L, mode, pbuf, g, b, s);
            else lattice_launch_t<double, false, false>(L, mode, pbuf, g, b, s);
        }
    } else {
        if (odd) {
            if (record) lattice_launch_t<float, true, true>(L, mode, pbuf, g, b, s);
            else lattice_launch_t<float, true, false>(L, mode, pbuf, g, b, s);
        } else {
            if (record) lattice_launch_t<float, false, true>(L, mode, pbuf, g, b, s);
            else lattice_launch_t<float, false, false>(L, mode, pbuf, g, b, s);
        }
    }
    return cudaGetLastError();
}

template <typename T, bool PER>
static cudaError_t near_t(const LbView &L, bool odd, bool record, int pbuf, cudaStream_t s, int prio)
{
    const dim3 g(2 * 152), b(256);  // grid-stride over the patch box
    if (odd) {
        if (record) return launch_p(k_lattice_near<T, true, true, PER>, g, b, s, prio, L, pbuf);
        return launch_p(k_lattice_near<T, true, false, PER>, g, b, s, prio, L, pbuf);
    }
    if (record) return launch_p(k_lattice_near<T, false, true, PER>, g, b, s, prio, L, pbuf);
    return launch_p(k_lattice_near<T, false, false, PER>, g, b, s, prio, L, pbuf);
}

cudaError_t launch_near(const LbView &L, bool odd, bool record, int pbuf, cudaStream_t s, int prio)
{
    const bool per = any_periodic(L);
    if (L.precision == IBL_FP64)
        return per ? near_t<double, true>(L, odd, record, pbuf, s, prio) : near_t<double, false>(L, odd, record, pbuf, s, prio);
    return per ? near_t<float, true>(L, odd, record, pbuf, s, prio) : near_t<float, false>(L, odd, record, pbuf, s, prio);
}

template <typename T>
__global__ void k_convert_frames(LbView L, int k0, int k1)
{
    const int i = 9 * k0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 9 * k1) static_cast<T *>(const_cast<void *>(L.frames_t))[i] = T(L.frames[i]);
}

cudaError_t launch_convert_frames(const LbView &L, int k0, int k1, cudaStream_t s)
{
    const unsigned g = blocks_for(9LL * (k1 - k0), 256);
    if (L.precision == IBL_FP64) k_convert_frames<double><<<g, 256, 0, s>>>(L, k0, k1);
    else k_convert_frames<float><<<g, 256, 0, s>>>(L, k0, k1);
    return cudaGetLastError();
}

// Lanes per mesh node of a single droplet's force/spread and interpolation
// kernels.  A small mesh (one 16-lane block per SM or fewer) takes 16 lanes:
// its step is the droplet chain's latency, and more, shorter threads shorten
// it.  A larger mesh takes kFwdLanes: there the lattice update sets the step,
// and half the threads hold half the SM slots the chain takes from it.
static int fwd_lanes(const MeshView &M)
{
    return (long long)M.nv * 16 <= (long long)sm_count() * kIbThreads ? 16 : kFwdLanes;
}

// Blocks of the single droplet's node-group kernels: one per group of
// nodes.  (The kernels are block-strided, so a grid may be capped; capped at
// two blocks per SM, the 256^3 step took 431 instead of 437 us and the 200^3
// step without regularisation 218.6 instead of 223.0 us, but the 200^3 step
// regularised after every step 254 instead of 235 us: the longer droplet
// chain then no longer fits beside the outside update.)
static unsigned ib_grid(int nblk) { return (unsigned)nblk; }

cudaError_t launch_spread(const LbView &L, const MeshView &M, int next_buf, cudaStream_t s, int prio)
{
    const int lanes = fwd_lanes(M);
    const int nblk = (int)blocks_for((long long)M.nv * lanes, kIbThreads);
    const dim3 g(ib_grid(nblk)), b(kIbThreads);
    if (lanes == 16) {
        if (L.precision == IBL_FP64) return launch_p(k_spread<double, 16>, g, b, s, prio, L, M, next_buf, nblk);
        return launch_p(k_spread<float, 16>, g, b, s, prio, L, M, next_buf, nblk);
    }
    if (L.precision == IBL_FP64) return launch_p(k_spread<double, kFwdLanes>, g, b, s, prio, L, M, next_buf, nblk);
    return launch_p(k_spread<float, kFwdLanes>, g, b, s, prio, L, M, next_buf, nblk);
}

cudaError_t launch_centre(const LbView &L, const MeshView &M, int buf, cudaStream_t s, int prio)
{
    return launch_p(k_centre, dim3(kCentreBlocks), dim3(kCentreThreads), s, prio, L, M, buf);
}

cudaError_t launch_indicator(const LbView &L, const MeshView &M, int buf, cudaStream_t s, int prio)
{
    return launch_p(k_indicator, dim3(blocks_for(M.nt, 128)), dim3(128), s, prio, L, M, buf);
}

cudaError_t launch_interp(const LbView &L, const MeshView &M, cudaStream_t s, int prio)
{
    const int lanes = fwd_lanes(M);
    const int nblk = (int)blocks_for((long long)M.nv * lanes, kIbThreads);
    const dim3 g(ib_grid(nblk)), b(kIbThreads);
    if (lanes == 16) {
        if (L.precision == IBL_FP64) return launch_p(k_interp<double, 16>, g, b, s, prio, L, M, nblk);
        return launch_p(k_interp<float, 16>, g, b, s, prio, L, M, nblk);
    }
    if (L.precision == IBL_FP64) return launch_p(k_interp<double, kFwdLanes>, g, b, s, prio, L, M, nblk);
    return launch_p(k_interp<float, kFwdLanes>, g, b, s, prio, L, M, nblk);
}

cudaError_t launch_regularize(const LbView &L, const MeshView &M, const RegParams &p, int buf, cudaStream_t s,
                              int prio)
{
    // a cluster of one CTA per SM when the mesh fits (and the device takes
    // the cluster size), the single-CTA kernel otherwise
    static int cluster_ok = -1;
    if (cluster_ok < 0) {
        cluster_ok = 0;
        cudaError_t e = cudaFuncSetAttribute(k_regularize_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_regularize_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(double) * (12 * kRegPerCta + 8)));
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(kRegCluster);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = sizeof(double) * (12 * kRegPerCta + 8);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = kRegCluster;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            e = cudaOccupancyMaxActiveClusters(&n, k_regularize_cluster, &cfg);
            if (e == cudaSuccess && n > 0) cluster_ok = 1;
        }
        cudaGetLastError();  // a refused attribute only selects the fallback
    }
    if (!cluster_ok || M.nv > kRegCluster * kRegPerCta)
        return launch_p(k_regularize, dim3(1), dim3(1024), s, prio, L, M, p, buf);
    const int P = (M.nv + kRegCluster - 1) / kRegCluster;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kRegCluster);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = sizeof(double) * (12 * (size_t)P + 8);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kRegCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributePriority;
    at[1].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = prio != 0 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_regularize_cluster, L, M, p, buf, P);
}

cudaError_t launch_observables(const LbView &L, const MeshView &M, cudaStream_t s, int prio)
{
    int g = (M.nt + 255) / 256;
    if (g > kObsBlocksMax) g = kObsBlocksMax;
    return launch_p(k_observables, dim3(g), dim3(256), s, prio, L, M);
}

cudaError_t launch_patch_from_mesh(const LbView &L, const MeshView &M, int buf, cudaStream_t s)
{
    k_patch<<<1, 256, 0, s>>>(L, M, buf);
    return cudaGetLastError();
}

// Ensemble phases.  Each launches one kernel per group of up to kGroup
// members; the group's views travel in the kernel parameters.
namespace {
struct Groups {
    // parameter blocks are large: kept off the stack
    LbGroup lg;
    MeshGroup mg;
};
Groups &groups()
{
    static thread_local Groups g;
    return g;
}
void fill_group(const EnsembleView &E, int m0, int m1)
{
    Groups &G = groups();
    for (int k = m0; k < m1; ++k) {
        G.lg.v[k - m0] = E.lv[k];
        G.mg.v[k - m0] = E.mv[k];
    }
}
}  // namespace

static int ens_shape(const EnsembleView &E) { return E.shape >= 0 && E.shape < kEnsShapes ? E.shape : kEnsDefaultShape; }

// Blocks of a batched droplet-side kernel over nb node groups: all of them,
// or, in the capped shapes, at most the shape's cap per SM (the kernels then
// stride over the node groups).
static int chain_grid(const EnsembleView &E, int nb)
{
    if (!ens_shape_capped(ens_shape(E))) return nb;
    const int cap = ens_shape_cap(ens_shape(E)) * sm_count();
    return nb < cap ? nb : cap;
}

template <class P>
static cudaError_t ensemble_pre_t(const EnsembleView &E, int m0, int m1, int pbuf, int nxt, cudaStream_t s, int prio)
{
    Groups &G = groups();
    bool recentre = false;
    int nt_max = 0;
    for (int k = m0; k < m1; ++k) {
        recentre = recentre || E.lv[k].recentre != 0;
        nt_max = E.mv[k].nt > nt_max ? E.mv[k].nt : nt_max;
    }
    cudaError_t e = cudaSuccess;
    if (recentre)
        e = launch_p(k_centre_batched, dim3(kCentreBlocks, m1 - m0), dim3(kCentreThreads), s, prio, G.lg, G.mg, pbuf);
    int tb = (nt_max + 127) / 128;
    if (ens_shape_capped(ens_shape(E))) {
        const int cap = ens_shape_cap(ens_shape(E)) * sm_count() / (m1 - m0);
        tb = tb < cap ? tb : (cap < 1 ? 1 : cap);
    }
    if (e == cudaSuccess) e = launch_p(k_tri_moment_batched<P>, dim3(tb, m1 - m0), dim3(128), s, prio, G.mg);
    const int nb0 = E.node_start[m0], nb = E.node_start[m1] - nb0;
    const dim3 g(chain_grid(E, nb));
    if (e == cudaSuccess) {
        if (E.precision == IBL_FP64)
            e = launch_p(k_spread_batched<double, P>, g, dim3(kIbThreads), s, prio, G.lg, G.mg, m0, nb0, nb,
                         E.node_member, E.node_start_d, nxt);
        else
            e = launch_p(k_spread_batched<float, P>, g, dim3(kIbThreads), s, prio, G.lg, G.mg, m0, nb0, nb,
                         E.node_member, E.node_start_d, nxt);
    }
    return e;
}

cudaError_t launch_ensemble_pre(const EnsembleView &E, long long step, cudaStream_t s, int prio)
{
    const int pbuf = (int)(step % 3), nxt = (int)((step + 1) % 3);
    const int n = (int)E.lv.size();
    const bool keep = ens_shape_keep(ens_shape(E));
    for (int m0 = 0; m0 < n; m0 += kGroup) {
        const int m1 = m0 + kGroup < n ? m0 + kGroup : n;
        fill_group(E, m0, m1);
        const cudaError_t e = keep ? ensemble_pre_t<L2Keep>(E, m0, m1, pbuf, nxt, s, prio)
                                   : ensemble_pre_t<L2Plain>(E, m0, m1, pbuf, nxt, s, prio);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T, bool PER, class P>
static cudaError_t ensemble_near_t(const EnsembleView &E, bool odd, int m0, int m1, int pbuf, cudaStream_t s, int prio)
{
    Groups &G = groups();
    // blocks per member: kEnsNearBlocks, or in the capped shapes about the
    // shape's cap per SM over the whole group
    int per = kEnsNearBlocks;
    if (ens_shape_capped(ens_shape(E))) {
        per = ens_shape_cap(ens_shape(E)) * sm_count() / (m1 - m0);
        per = per < 1 ? 1 : (per > kEnsNearBlocks ? kEnsNearBlocks : per);
    }
    const dim3 g(per, m1 - m0), b(256);
    return odd ? launch_p(k_lattice_near_batched<T, true, PER, P>, g, b, s, prio, G.lg, pbuf)
               : launch_p(k_lattice_near_batched<T, false, PER, P>, g, b, s, prio, G.lg, pbuf);
}

template <class P>
static cudaError_t ensemble_near_p(const EnsembleView &E, bool odd, int m0, int m1, int pbuf, cudaStream_t s,
                                   int prio)
{
    bool per = false;
    for (int k = m0; k < m1; ++k) per = per || any_periodic(E.lv[k]);
    if (E.precision == IBL_FP64)
        return per ? ensemble_near_t<double, true, P>(E, odd, m0, m1, pbuf, s, prio)
                   : ensemble_near_t<double, false, P>(E, odd, m0, m1, pbuf, s, prio);
    return per ? ensemble_near_t<float, true, P>(E, odd, m0, m1, pbuf, s, prio)
               : ensemble_near_t<float, false, P>(E, odd, m0, m1, pbuf, s, prio);
}

cudaError_t launch_ensemble_near(const EnsembleView &E, long long step, cudaStream_t s, int prio)
{
    const bool odd = (step & 1) != 0;
    const int pbuf = (int)(step % 3);
    const int n = (int)E.lv.size();
    const bool keep = ens_shape_keep(ens_shape(E));
    for (int m0 = 0; m0 < n; m0 += kGroup) {
        const int m1 = m0 + kGroup < n ? m0 + kGroup : n;
        fill_group(E, m0, m1);
        const cudaError_t e = keep ? ensemble_near_p<L2Keep>(E, odd, m0, m1, pbuf, s, prio)
                                   : ensemble_near_p<L2Plain>(E, odd, m0, m1, pbuf, s, prio);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T, bool ODD, bool PER>
static void far_batched_t(const EnsembleView &E, int m0, int pbuf, int waves, int ti, cudaStream_t s)
{
    const int m1 = m0 + kGroup < (int)E.lv.size() ? m0 + kGroup : (int)E.lv.size();
    const int lb0 = E.lat_start[ti][m0], lbn = E.lat_start[ti][m1] - lb0;
    const int nt = ti == 0 ? 128 : 256;
    const int per_sm = (sizeof(T) == 4 ? 1024 : 512) / nt;
    const int ahead = waves * sm_count() * per_sm * nt;
    Groups &G = groups();
    if (nt == 128)
        k_lattice_batched<T, ODD, 128, PER><<<lbn, 128, 0, s>>>(G.lg, m0, lb0, E.lat_member[ti], E.lat_start_d[ti], pbuf, ahead);
    else
        k_lattice_batched<T, ODD, 256, PER><<<lbn, 256, 0, s>>>(G.lg, m0, lb0, E.lat_member[ti], E.lat_start_d[ti], pbuf, ahead);
}

cudaError_t launch_ensemble_far(const EnsembleView &E, long long step, cudaStream_t s)
{
    const bool odd = (step & 1) != 0;
    const int pbuf = (int)(step % 3);
    const int n = (int)E.lv.size();
    const int shape = ens_shape(E);
    const int ti = ens_shape_threads(shape) == 128 ? 0 : 1, waves = ens_shape_waves(shape);
    for (int m0 = 0; m0 < n; m0 += kGroup) {
        const int m1 = m0 + kGroup < n ? m0 + kGroup : n;
        fill_group(E, m0, m1);
        bool per = false;
        for (int k = m0; k < m1; ++k) per = per || any_periodic(E.lv[k]);
        if (E.precision == IBL_FP64) {
            if (per) {
                if (odd) far_batched_t<double, true, true>(E, m0, pbuf, waves, ti, s);
                else far_batched_t<double, false, true>(E, m0, pbuf, waves, ti, s);
            } else {
                if (odd) far_batched_t<double, true, false>(E, m0, pbuf, waves, ti, s);
                else far_batched_t<double, false, false>(E, m0, pbuf, waves, ti, s);
            }
        } else {
            if (per) {
                if (odd) far_batched_t<float, true, true>(E, m0, pbuf, waves, ti, s);
                else far_batched_t<float, false, true>(E, m0, pbuf, waves, ti, s);
            } else {
                if (odd) far_batched_t<float, true, false>(E, m0, pbuf, waves, ti, s);
                else far_batched_t<float, false, false>(E, m0, pbuf, waves, ti, s);
            }
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ensemble_interp(const EnsembleView &E, cudaStream_t s, int prio)
{
    const int n = (int)E.lv.size();
    const bool keep = ens_shape_keep(ens_shape(E));
    Groups &G = groups();
    for (int m0 = 0; m0 < n; m0 += kGroup) {
        const int m1 = m0 + kGroup < n ? m0 + kGroup : n;
        fill_group(E, m0, m1);
        const int nb0 = E.node_start[m0], nb = E.node_start[m1] - nb0;
        const dim3 g(chain_grid(E, nb)), b(kIbThreads);
        cudaError_t e;
        if (E.precision == IBL_FP64)
            e = keep ? launch_p(k_interp_batched<double, L2Keep>, g, b, s, prio, G.lg, G.mg, m0, nb0, nb,
                                E.node_member, E.node_start_d)
                     : launch_p(k_interp_batched<double, L2Plain>, g, b, s, prio, G.lg, G.mg, m0, nb0, nb,
                                E.node_member, E.node_start_d);
        else
            e = keep ? launch_p(k_interp_batched<float, L2Keep>, g, b, s, prio, G.lg, G.mg, m0, nb0, nb,
                                E.node_member, E.node_start_d)
                     : launch_p(k_interp_batched<float, L2Plain>, g, b, s, prio, G.lg, G.mg, m0, nb0, nb,
                                E.node_member, E.node_start_d);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_observables_batched(const EnsembleView &E, const std::vector<char> &due, cudaStream_t s, int prio)
{
    const int n = (int)E.lv.size();
    Groups &G = groups();
    for (int m0 = 0; m0 < n; m0 += kGroup) {
        const int m1 = m0 + kGroup < n ? m0 + kGroup : n;
        unsigned long long mask = 0;
        int nt_max = 0;
        for (int k = m0; k < m1; ++k)
            if (due[k]) {
                mask |= 1ull << (k - m0);
                nt_max = E.mv[k].nt > nt_max ? E.mv[k].nt : nt_max;
            }
        if (!mask) continue;
        fill_group(E, m0, m1);
        int g = (nt_max + 255) / 256;
        if (g > kObsBlocksMax) g = kObsBlocksMax;
        const cudaError_t e =
            launch_p(k_observables_batched, dim3(g, m1 - m0), dim3(256), s, prio, G.lg, G.mg, mask);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void velocity_table(int c[19][3], double w[19])
{
    for (int i = 0; i < 19; ++i) {
        c[i][0] = cxf(i);
        c[i][1] = cyf(i);
        c[i][2] = czf(i);
        w[i] = wgt(i);
    }
}

}  // namespace iblb

// ---------------------------------------------------------------------------
// Allocation-free mesh regularisation.
//
// Some callers cannot allocate device memory: a host program whose own
// allocator has reserved the device's memory up front (so any other
// allocation fails or fragments its pool), a control loop with a fixed time
// budget that cannot absorb an allocation call that may synchronise the
// device, or a plug-in whose host forbids it to allocate.  For them this
// variant of the regularisation kernel keeps its scratch in a fixed array
// of this file instead of in a caller workspace.  The array is part of the
// library image, so every GPU that loads the library holds it (1.18 MB)
// until the process exits.
namespace iblb {
namespace {

constexpr int kNoAllocMaxNodes = 16384;  // enough for a level-5 icosphere (10242 nodes)

// x_o, the ping-pong iterate and x_b, each [kNoAllocMaxNodes][3] doubles.
static __device__ __align__(256) double g_noalloc_scratch[3 * 3 * kNoAllocMaxNodes];

// Same iteration as k_regularize (Sec. 3.3), reading and writing only the
// caller's positions and the static scratch; result[0] = iterations,
// result[1] = 1 if the exit test held.
__global__ void __launch_bounds__(1024)
    k_regularize_noalloc(double *r, const int *nb_ptr, const int *nb_idx, int nv, double *scratch, RegParams p,
                         int *result)
{
    __shared__ double sh[32];
    double *xo = scratch, *s1 = scratch + 3 * kNoAllocMaxNodes, *xb = scratch + 6 * kNoAllocMaxNodes;
    double *buf[2] = {r, s1};
    for (int i = threadIdx.x; i < 3 * nv; i += blockDim.x) xo[i] = r[i];
    __syncthreads();
    const double sg = p.plus_sign ? 1.0 : -1.0;
    int cur = 0, it = 0;
    bool conv = false;
    while (it < p.max_iter) {
        ++it;
        const double *xq = buf[cur];
        double *xp = buf[cur ^ 1];
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            const int b0 = nb_ptr[i], b1 = nb_ptr[i + 1];
            const int ni = b1 - b0;
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = b0; k < b1; ++k) s += xq[3 * nb_idx[k] + a];
                const double v = p.alpha * xo[3 * i + a] + (1.0 - p.alpha) / ni * s;
                xp[3 * i + a] = v;
                xb[3 * i + a] = v - (p.alpha * xo[3 * i + a] + (1.0 - p.alpha) * xq[3 * i + a]);
            }
        }
        __syncthreads();
        double dmax = 0.0;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            const int b0 = nb_ptr[i], b1 = nb_ptr[i + 1];
            const int ni = b1 - b0;
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = b0; k < b1; ++k) s += xb[3 * nb_idx[k] + a];
                const double v = xp[3 * i + a] - (p.gamma * xb[3 * i + a] + sg * (1.0 - p.gamma) / ni * s);
                xp[3 * i + a] = v;
                const double d = v - xq[3 * i + a];
                d2 += d * d;
            }
            dmax = fmax(dmax, sqrt(d2));
        }
        dmax = block_max(dmax, sh);
        cur ^= 1;
        if (dmax < p.tol) {
            conv = true;
            break;
        }
    }
    if (cur != 0) {
        for (int i = threadIdx.x; i < 3 * nv; i += blockDim.x) r[i] = s1[i];
    }
    if (threadIdx.x == 0) {
        result[0] = it;
        result[1] = conv ? 1 : 0;
    }
}

// Device address of the array per device ordinal, with the id of the
// context it was looked up in: the array is part of the module loaded into
// that context, so another context (a driver-API context made current, or the
// primary context created anew after cudaDeviceReset) holds it elsewhere.
struct NoAllocSlot {
    unsigned long long ctx_id;
    double *ptr;
};
std::mutex g_noalloc_mu;
NoAllocSlot g_noalloc_slot[256] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 if there is none yet).
// Called with g_noalloc_mu held.
cudaError_t current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    *id = 0;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess) return e;
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(a);
        get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS) return cudaErrorUnknown;
    if (!c) return cudaSuccess;
    return get_id(c, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace
}  // namespace iblb

extern "C" int ibl_regularize_noalloc(double *r, const int32_t *nb_ptr, const int32_t *nb_idx, int n_nodes,
                                      double alpha, double gamma, double tol, int max_iter, int plus_sign,
                                      int32_t *result, void *stream)
{
    using namespace iblb;
    if (!r || !nb_ptr || !nb_idx || !result) return iblb_set_error(IBL_EINVAL, "null pointer argument");
    if (n_nodes < 1 || n_nodes > kNoAllocMaxNodes)
        return iblb_set_error(IBL_EINVAL, "ibl_regularize_noalloc: n_nodes must be in 1..16384 (the size of its "
                                          "fixed scratch array)");
    if (!(alpha >= 0 && alpha <= 1) || !(gamma >= 0 && gamma <= 1) || !(tol > 0) || max_iter < 1)
        return iblb_set_error(IBL_EINVAL, "regularisation parameters out of range");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return iblb_set_error(IBL_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return iblb_set_error(IBL_EINVAL, "device ordinal out of range");
    double *scratch = nullptr;
    {
        // first call on this device, or first call in another context of
        // it: look up the array's device address with the device current
        // (the name alone is a host-side stand-in, not a device address)
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        unsigned long long ctx = 0;
        e = current_context_id(&ctx);
        if (e != cudaSuccess) return iblb_set_error(IBL_ECUDA, cudaGetErrorString(e));
        NoAllocSlot &slot = g_noalloc_slot[dev];
        if (ctx == 0 || !slot.ptr || slot.ctx_id != ctx) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // also creates the context if there is none yet
            if (e != cudaSuccess) return iblb_set_error(IBL_ECUDA, cudaGetErrorString(e));
            e = current_context_id(&ctx);
            if (e != cudaSuccess) return iblb_set_error(IBL_ECUDA, cudaGetErrorString(e));
            slot.ptr = static_cast<double *>(p);
            slot.ctx_id = ctx;
        }
        scratch = slot.ptr;
    }
    RegParams p{alpha, gamma, tol, max_iter, plus_sign ? 1 : 0};
    k_regularize_noalloc<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(
        r, reinterpret_cast<const int *>(nb_ptr), reinterpret_cast<const int *>(nb_idx), n_nodes, scratch, p,
        reinterpret_cast<int *>(result));
    e = cudaGetLastError();
    if (e != cudaSuccess) return iblb_set_error(IBL_ECUDA, cudaGetErrorString(e));
    return IBL_OK;
}
