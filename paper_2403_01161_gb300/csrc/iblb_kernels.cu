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
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <utility>

#include "iblb_internal.h"

namespace iblb {
namespace {

// ---------------------------------------------------------------------------
// D3Q19 velocity set, library order: rest, nine "positive" links, then their
// opposites at i + 9.  Weights 1/3, 1/18, 1/36 (Sec. 3.1).
__host__ __device__ constexpr int cxf(int i)
{
    const int t[19] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, -1, 0, 0, -1, -1, -1, -1, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cyf(int i)
{
    const int t[19] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 0, -1, 0, -1, 1, 0, 0, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int czf(int i)
{
    const int t[19] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1};
    return t[i];
}

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
__host__ __device__ constexpr int c2(int i) { return cxf(i) * cxf(i) + cyf(i) * cyf(i) + czf(i) * czf(i); }
__host__ __device__ constexpr int comp(int i, int a) { return a == 0 ? cxf(i) : (a == 1 ? cyf(i) : czf(i)); }
__host__ __device__ constexpr double wgt(int i) { return c2(i) == 0 ? 1.0 / 3.0 : (c2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0); }

template <int... Is, class F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, Is...>, F &&f)
{
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

// ---------------------------------------------------------------------------
// Box boundary (Sec. 3.1).  SX, SY, SZ = -1 on the plane l = 0, +1 on l = L,
// 0 elsewhere.  Population j is unknown when its source x - c_j is outside.
template <int SX, int SY, int SZ>
__host__ __device__ constexpr bool unknown_dir(int j)
{
    return (SX != 0 && cxf(j) * SX < 0) || (SY != 0 && cyf(j) * SY < 0) || (SZ != 0 && czf(j) * SZ < 0);
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
        constexpr int E = SX == 0 ? 0 : (SY == 0 ? 1 : 2);
        constexpr int PE = E + 1, ME = E + 10;  // +e_E and -e_E in the library order
        static_assert(comp(PE, E) == 1 && comp(ME, E) == -1, "axis links");
        const T dE = f[PE] - f[ME];
        const bool wall = (rule == IBL_EDGE_PAPER_PLUS_WALL);
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && !unknown_dir<SX, SY, SZ>(opp(j))) {
                constexpr int i = opp(j);
                T v = f[i];
                if constexpr (comp(i, E) != 0) v -= T(0.25) * T(comp(i, E)) * dE;
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
            if constexpr (i != 0 && !(unknown_dir<SX, SY, SZ>(i) && unknown_dir<SX, SY, SZ>(opp(i)))) sb += f[i];
        });
        const T fb = sb * T(1.0 / 22.0);
        sfor<19>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr (j != 0 && unknown_dir<SX, SY, SZ>(j) && unknown_dir<SX, SY, SZ>(opp(j))) f[j] = fb;
        });
        f[0] = T(12) * fb;
    } else if constexpr (NB == 3) {
        // Corner, Eq. (zh-buried-links-corners); non-buried unknowns take
        // (moving-wall) bounce-back; f_0 = 12 f_b.
        const bool wall = (rule == IBL_EDGE_PAPER_PLUS_WALL);
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
            if constexpr (j != 0 && cs == 0) f[j] = fb;
        });
        f[0] = T(12) * fb;
    }
}

template <typename T>
__device__ __noinline__ void bc_dispatch(T (&f)[19], const T (&uw)[3], int rule, int code)
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

__device__ __forceinline__ const double *frame_ptr(const LbView &L, long long step)
{
    long long k = step / L.n_hold;
    if (k > L.n_frames - 1) k = L.n_frames - 1;
    return L.frames + 9 * k;
}

// Neighbour coordinate along one axis: x + d (d in {-1,0,1}); periodic axes
// wrap, Zou-He axes return -1 outside the box.
__device__ __forceinline__ int step_coord(int x, int d, int n, bool periodic)
{
    int y = x + d;
    if (periodic) {
        if (y < 0) y += n;
        else if (y >= n) y -= n;
        return y;
    }
    return (y < 0 || y >= n) ? -1 : y;
}

// ---------------------------------------------------------------------------
// Lattice update: streaming (AA pattern) + boundary rebuild + moments with
// half-force momentum + BGK + Guo source, Eqs. (LBMEQ)-(density_velocity_LB).
template <typename T, bool ODD, bool REC>
__global__ void __launch_bounds__(256) k_lattice(LbView L)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = node < L.nodes;
    int x = 0, y = 0, z = 0;
    if (active) {
        const int nxy = nx * ny;
        z = node / nxy;
        const int rem = node - z * nxy;
        y = rem / nx;
        x = rem - y * nx;
    }
    T *__restrict__ f = static_cast<T *>(L.f);
    const long long qs = L.qs;
    bool bad = false;
    if (active) {
        const bool px = L.bc[0] == IBL_BC_PERIODIC, py = L.bc[1] == IBL_BC_PERIODIC,
                   pz = L.bc[2] == IBL_BC_PERIODIC;
        const int sx = px ? 0 : (x == 0 ? -1 : (x == nx - 1 ? 1 : 0));
        const int sy = py ? 0 : (y == 0 ? -1 : (y == ny - 1 ? 1 : 0));
        const int sz = pz ? 0 : (z == 0 ? -1 : (z == nz - 1 ? 1 : 0));
        const int xm = step_coord(x, -1, nx, px), xp = step_coord(x, 1, nx, px);
        const int ym = step_coord(y, -1, ny, py), yp = step_coord(y, 1, ny, py);
        const int zm = step_coord(z, -1, nz, pz), zp = step_coord(z, 1, nz, pz);

        T g[19];
        if constexpr (!ODD) {
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                g[i] = f[i * qs + node];
            });
        } else {
            // source x - c_i, slot opp(i)
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const int ax = cxf(i) == 0 ? x : (cxf(i) > 0 ? xm : xp);
                const int ay = cyf(i) == 0 ? y : (cyf(i) > 0 ? ym : yp);
                const int az = czf(i) == 0 ? z : (czf(i) > 0 ? zm : zp);
                if (ax >= 0 && ay >= 0 && az >= 0)
                    g[i] = f[opp(i) * qs + (ax + nx * (ay + ny * az))];
                else
                    g[i] = T(0);
            });
        }

        if (sx | sy | sz) {
            const double *A = frame_ptr(L, L.ctl->step);
            const double lx = x - 0.5 * (nx - 1), ly = y - 0.5 * (ny - 1), lz = z - 0.5 * (nz - 1);
            const T uw[3] = {T(A[0] * lx + A[1] * ly + A[2] * lz), T(A[3] * lx + A[4] * ly + A[5] * lz),
                             T(A[6] * lx + A[7] * ly + A[8] * lz)};
            bc_dispatch<T>(g, uw, L.rule, (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1));
        }

        // droplet patch: read the spread force (and clear it), store u below
        bool in_patch = false;
        {
            const Ctl *c = L.ctl;
            int dx = x - c->patch_lo[0], dy = y - c->patch_lo[1], dz = z - c->patch_lo[2];
            if (px && dx < 0) dx += nx;
            if (py && dy < 0) dy += ny;
            if (pz && dz < 0) dz += nz;
            in_patch = dx >= 0 && dx <= c->patch_ext[0] && dy >= 0 && dy <= c->patch_ext[1] && dz >= 0 &&
                       dz <= c->patch_ext[2];
        }
        T Fx = T(0), Fy = T(0), Fz = T(0);
        T *__restrict__ force = static_cast<T *>(L.force);
        const int nodes = L.nodes;
        if (in_patch) {
            Fx = force[node];
            Fy = force[nodes + node];
            Fz = force[2 * nodes + node];
            force[node] = T(0);
            force[nodes + node] = T(0);
            force[2 * nodes + node] = T(0);
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
        const T ux = (jx + T(0.5) * Fx) * ir, uy = (jy + T(0.5) * Fy) * ir, uz = (jz + T(0.5) * Fz) * ir;
        const T uu = ux * ux + uy * uy + uz * uz;
        bad = !(uu <= T(0.09)) || !(drho == drho);
        const T om = T(L.omega);
        const T fpre = T(1) - T(0.5) * om;
        const T uF = ux * Fx + uy * Fy + uz * Fz;
        const T base = T(1.5) * uu;
        sfor<19>([&](auto I) {
            constexpr int i = decltype(I)::value;
            T cu = T(0), cF = T(0);
            if constexpr (cxf(i) != 0) { cu += T(cxf(i)) * ux; cF += T(cxf(i)) * Fx; }
            if constexpr (cyf(i) != 0) { cu += T(cyf(i)) * uy; cF += T(cyf(i)) * Fy; }
            if constexpr (czf(i) != 0) { cu += T(czf(i)) * uz; cF += T(czf(i)) * Fz; }
            constexpr double w = wgt(i);
            const T geq = T(w) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - base));
            const T src = fpre * T(w) * (T(3) * (cF - uF) + T(9) * cu * cF);
            g[i] = g[i] + om * (geq - g[i]) + src;
        });

        if constexpr (!ODD) {
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                f[opp(i) * qs + node] = g[i];
            });
        } else {
            // destination x + c_i, slot i
            sfor<19>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const int ax = cxf(i) == 0 ? x : (cxf(i) > 0 ? xp : xm);
                const int ay = cyf(i) == 0 ? y : (cyf(i) > 0 ? yp : ym);
                const int az = czf(i) == 0 ? z : (czf(i) > 0 ? zp : zm);
                if (ax >= 0 && ay >= 0 && az >= 0) f[i * qs + (ax + nx * (ay + ny * az))] = g[i];
            });
        }
        if (in_patch) {
            T *__restrict__ vel = static_cast<T *>(L.vel);
            vel[node] = ux;
            vel[nodes + node] = uy;
            vel[2 * nodes + node] = uz;
        }
        if constexpr (REC) {
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
    // sticky instability flag, one atomic per warp at most
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m != 0u && (threadIdx.x & 31) == 0) atomicOr(&L.ctl->err, IBL_ERRBIT_UNSTABLE);
    // the last block to finish advances the step counter
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&L.ctl->lb_blocks_done, 1u);
        if (t == gridDim.x - 1) {
            L.ctl->step += 1;
            L.ctl->lb_blocks_done = 0u;
            __threadfence();
        }
    }
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
__device__ __forceinline__ double peskin_phi(double x)
{
    const double a = fabs(x);
    if (a < 1.0) return 0.125 * (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a));
    if (a < 2.0) return 0.125 * (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
    return 0.0;
}

// The four stencil nodes floor(r)-1 .. floor(r)+2 along one axis and their
// weights; on a Zou-He axis all must be interior nodes (1..n-2), periodic
// axes wrap.  Returns false for an invalid stencil (the caller flags it).
__device__ __forceinline__ bool stencil(double ra, int n, bool periodic, int idx[4], double w[4])
{
    if (!(fabs(ra) < 1e8)) return false;
    const int base = (int)floor(ra) - 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int g = base + k;
        w[k] = peskin_phi(ra - (double)g);
        if (periodic) {
            g %= n;
            if (g < 0) g += n;
        } else if (g < 1 || g > n - 2) {
            return false;
        }
        idx[k] = g;
    }
    return true;
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Nodal force F_i = -sigma dA/dx_i (Eq. (pi_drop)) gathered over the
// triangles around node i, then spread with the 4-point delta
// (Eq. (ibm_force_d)(a)) by atomic adds into the Eulerian force.
template <typename T>
__global__ void __launch_bounds__(128) k_spread(LbView L, MeshView M)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M.nv) return;
    double F[3] = {0.0, 0.0, 0.0};
    for (int k = M.n2t_ptr[i]; k < M.n2t_ptr[i + 1]; ++k) {
        const int e = M.n2t[k];
        const int t = e / 3, slot = e - 3 * t;
        const int v0 = M.tris[3 * t], v1 = M.tris[3 * t + 1], v2 = M.tris[3 * t + 2];
        const double x0[3] = {M.r[3 * v0], M.r[3 * v0 + 1], M.r[3 * v0 + 2]};
        const double x1[3] = {M.r[3 * v1], M.r[3 * v1 + 1], M.r[3 * v1 + 2]};
        const double x2[3] = {M.r[3 * v2], M.r[3 * v2 + 1], M.r[3 * v2 + 2]};
        double e1[3], e2[3], N[3];
        for (int a = 0; a < 3; ++a) { e1[a] = x1[a] - x0[a]; e2[a] = x2[a] - x0[a]; }
        cross3(e1, e2, N);
        const double len = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        const double n[3] = {N[0] / len, N[1] / len, N[2] / len};
        const double *xp = slot == 0 ? x1 : (slot == 1 ? x2 : x0);
        const double *xm = slot == 0 ? x2 : (slot == 1 ? x0 : x1);
        const double d[3] = {xm[0] - xp[0], xm[1] - xp[1], xm[2] - xp[2]};
        double g[3];
        cross3(n, d, g);
        for (int a = 0; a < 3; ++a) F[a] += -M.sigma * 0.5 * g[a];
    }
    M.fn[3 * i] = F[0];
    M.fn[3 * i + 1] = F[1];
    M.fn[3 * i + 2] = F[2];
    const double r[3] = {M.r[3 * i], M.r[3 * i + 1], M.r[3 * i + 2]};
    int ix[4], iy[4], iz[4];
    double wx[4], wy[4], wz[4];
    const bool ok = stencil(r[0], L.n[0], L.bc[0] == IBL_BC_PERIODIC, ix, wx) &&
                    stencil(r[1], L.n[1], L.bc[1] == IBL_BC_PERIODIC, iy, wy) &&
                    stencil(r[2], L.n[2], L.bc[2] == IBL_BC_PERIODIC, iz, wz);
    if (!ok) {
        atomicOr(&L.ctl->err, IBL_ERRBIT_WALL);
        return;
    }
    T *force = static_cast<T *>(L.force);
    const int nodes = L.nodes, nx = L.n[0], nxy = L.n[0] * L.n[1];
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b) {
            const int row = iy[b] * nx + iz[c] * nxy;
            for (int a = 0; a < 4; ++a) {
                const double dl = wx[a] * wy[b] * wz[c];
                const int id = row + ix[a];
                atomicAdd(force + id, T(F[0] * dl));
                atomicAdd(force + nodes + id, T(F[1] * dl));
                atomicAdd(force + 2 * nodes + id, T(F[2] * dl));
            }
        }
}

// order-preserving unsigned keys of doubles, for atomic min/max
__device__ __forceinline__ unsigned long long dkey(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k)
{
    const unsigned long long b = (k & 0x8000000000000000ull) ? (k & ~0x8000000000000000ull) : ~k;
    return __longlong_as_double((long long)b);
}

// Patch of lattice nodes the droplet's stencils can touch, from the node
// bounding box [mn, mx]: floor(mn)-1 .. floor(mx)+2 per axis.
__device__ void write_patch(const LbView &L, const double mn[3], const double mx[3])
{
    for (int a = 0; a < 3; ++a) {
        const int n = L.n[a];
        double lo_d = mn[a], hi_d = mx[a];
        if (!(lo_d > -1e8 && lo_d < 1e8) || !(hi_d > -1e8 && hi_d < 1e8) || hi_d < lo_d) {
            L.ctl->patch_lo[a] = 0;
            L.ctl->patch_ext[a] = n - 1;
            continue;
        }
        long long lo = (long long)floor(lo_d) - 1, hi = (long long)floor(hi_d) + 2;
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
        L.ctl->patch_lo[a] = (int)lo;
        L.ctl->patch_ext[a] = (int)(hi - lo);
    }
}

// u at r_i by the 4-point delta (Eq. (ibm_force_d)(b)) and forward Euler
// (Eq. (fwd_euler)); then the bounding box of the advected nodes sets the
// patch of the next step (last block).
template <typename T>
__global__ void __launch_bounds__(128) k_interp(LbView L, MeshView M)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double r[3] = {0.0, 0.0, 0.0};
    bool have = false;
    if (i < M.nv) {
        r[0] = M.r[3 * i];
        r[1] = M.r[3 * i + 1];
        r[2] = M.r[3 * i + 2];
        have = true;
        int ix[4], iy[4], iz[4];
        double wx[4], wy[4], wz[4];
        const bool ok = stencil(r[0], L.n[0], L.bc[0] == IBL_BC_PERIODIC, ix, wx) &&
                        stencil(r[1], L.n[1], L.bc[1] == IBL_BC_PERIODIC, iy, wy) &&
                        stencil(r[2], L.n[2], L.bc[2] == IBL_BC_PERIODIC, iz, wz);
        if (!ok) {
            atomicOr(&L.ctl->err, IBL_ERRBIT_WALL);
        } else {
            const T *vel = static_cast<const T *>(L.vel);
            const int nodes = L.nodes, nx = L.n[0], nxy = L.n[0] * L.n[1];
            double v[3] = {0.0, 0.0, 0.0};
            for (int c = 0; c < 4; ++c)
                for (int b = 0; b < 4; ++b) {
                    const int row = iy[b] * nx + iz[c] * nxy;
                    for (int a = 0; a < 4; ++a) {
                        const double dl = wx[a] * wy[b] * wz[c];
                        const int id = row + ix[a];
                        v[0] += (double)vel[id] * dl;
                        v[1] += (double)vel[nodes + id] * dl;
                        v[2] += (double)vel[2 * nodes + id] * dl;
                    }
                }
            r[0] += v[0];
            r[1] += v[1];
            r[2] += v[2];
            M.r[3 * i] = r[0];
            M.r[3 * i + 1] = r[1];
            M.r[3 * i + 2] = r[2];
        }
    }
    // block min / max of the new positions
    __shared__ double smn[3][4], smx[3][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        double mn = have ? r[a] : 1e300, mx = have ? r[a] : -1e300;
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            smn[a][warp] = mn;
            smx[a][warp] = mx;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int a = 0; a < 3; ++a) {
            double mn = smn[a][0], mx = smx[a][0];
            for (int w = 1; w < nw; ++w) {
                mn = fmin(mn, smn[a][w]);
                mx = fmax(mx, smx[a][w]);
            }
            atomicMin(&L.ctl->key_min[a], dkey(mn));
            atomicMax(&L.ctl->key_max[a], dkey(mx));
        }
        __threadfence();
        const unsigned t = atomicAdd(&L.ctl->ib_blocks_done, 1u);
        if (t == gridDim.x - 1) {
            __threadfence();
            double mn[3], mx[3];
            for (int a = 0; a < 3; ++a) {
                mn[a] = dkey_inv(*(volatile unsigned long long *)&L.ctl->key_min[a]);
                mx[a] = dkey_inv(*(volatile unsigned long long *)&L.ctl->key_max[a]);
                L.ctl->key_min[a] = ~0ull;
                L.ctl->key_max[a] = 0ull;
            }
            write_patch(L, mn, mx);
            L.ctl->ib_blocks_done = 0u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Single-block reductions.
template <int K>
__device__ void block_sum(double (&v)[K], double (*sh)[K])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < K; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w][k];
            sh[0][k] = s;
        }
    }
    __syncthreads();
    for (int k = 0; k < K; ++k) v[k] = sh[0][k];
    __syncthreads();
}

__device__ double block_max(double v, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = sh[0];
        for (int w = 1; w < nw; ++w) m = fmax(m, sh[w]);
        sh[0] = m;
    }
    __syncthreads();
    const double out = sh[0];
    __syncthreads();
    return out;
}

__device__ void block_bbox_patch(const LbView &L, const double *r, int nv)
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
    if (threadIdx.x == 0) write_patch(L, mn, mx);
}

// Mesh regularisation, Sec. 3.3, one block: x_o fixed, x_q the previous
// iterate, x_p the new one (ping-pong between r and s1), x_b in s2.
__global__ void __launch_bounds__(1024) k_regularize(LbView L, MeshView M, RegParams p)
{
    __shared__ double sh[32];
    const int nv = M.nv;
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
    block_bbox_patch(L, M.r, nv);
    if (threadIdx.x == 0) {
        L.ctl->reg_iters = it;
        if (!conv) atomicOr(&L.ctl->err, IBL_ERRBIT_NOCONV);
    }
}

__global__ void __launch_bounds__(256) k_patch(LbView L, MeshView M)
{
    block_bbox_patch(L, M.r, M.nv);
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations: each
// rotation J in the (p,q) plane with t = sgn(th)/(|th| + sqrt(th^2 + 1)),
// th = (a_qq - a_pp)/(2 a_pq), c = 1/sqrt(1 + t^2), s = t c, annihilates a_pq.
__device__ void jacobi3(double a[3][3], double lam[3], double v[3][3])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) v[r][c] = (r == c) ? 1.0 : 0.0;
    const double scale = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]) + 1e-300;
    for (int sweep = 0; sweep < 60; ++sweep) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        if (off <= 1e-17 * scale) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0;
            const int q = pq == 0 ? 1 : 2;
            const double apq = a[p][q];
            if (apq == 0.0) continue;
            const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.0;
            const int r = 3 - p - q;
            const double arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
            for (int k = 0; k < 3; ++k) {
                const double vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - s * vkq;
                v[k][q] = s * vkp + c * vkq;
            }
        }
    }
    for (int k = 0; k < 3; ++k) lam[k] = a[k][k];
}

// Shape record (Sec. 2): enclosed volume, centroid and second moment by
// signed tetrahedra (ref, a, b, c), S = (5/V) M, eigen-decomposition, Taylor
// D and beta of Eq. (beta).  One block.
__global__ void __launch_bounds__(512) k_observables(LbView L, MeshView M)
{
    __shared__ double sh3[16][3];
    __shared__ double sh11[16][11];
    double ref[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < M.nv; i += blockDim.x)
        for (int a = 0; a < 3; ++a) ref[a] += M.r[3 * i + a];
    block_sum<3>(ref, sh3);
    for (int a = 0; a < 3; ++a) ref[a] /= M.nv;
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
    block_sum<11>(acc, sh11);
    if (threadIdx.x != 0) return;
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

}  // namespace

// ---------------------------------------------------------------------------
// launchers
static inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_init(const LbView &L, cudaStream_t s)
{
    const unsigned g = blocks_for(L.nodes, 256);
    if (L.precision == IBL_FP64) k_init<double><<<g, 256, 0, s>>>(L);
    else k_init<float><<<g, 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_lattice(const LbView &L, bool odd, bool record, cudaStream_t s)
{
    const unsigned g = blocks_for(L.nodes, 256);
    if (L.precision == IBL_FP64) {
        if (odd) {
            if (record) k_lattice<double, true, true><<<g, 256, 0, s>>>(L);
            else k_lattice<double, true, false><<<g, 256, 0, s>>>(L);
        } else {
            if (record) k_lattice<double, false, true><<<g, 256, 0, s>>>(L);
            else k_lattice<double, false, false><<<g, 256, 0, s>>>(L);
        }
    } else {
        if (odd) {
            if (record) k_lattice<float, true, true><<<g, 256, 0, s>>>(L);
            else k_lattice<float, true, false><<<g, 256, 0, s>>>(L);
        } else {
            if (record) k_lattice<float, false, true><<<g, 256, 0, s>>>(L);
            else k_lattice<float, false, false><<<g, 256, 0, s>>>(L);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_spread(const LbView &L, const MeshView &M, cudaStream_t s)
{
    const unsigned g = blocks_for(M.nv, 128);
    if (L.precision == IBL_FP64) k_spread<double><<<g, 128, 0, s>>>(L, M);
    else k_spread<float><<<g, 128, 0, s>>>(L, M);
    return cudaGetLastError();
}

cudaError_t launch_interp(const LbView &L, const MeshView &M, cudaStream_t s)
{
    const unsigned g = blocks_for(M.nv, 128);
    if (L.precision == IBL_FP64) k_interp<double><<<g, 128, 0, s>>>(L, M);
    else k_interp<float><<<g, 128, 0, s>>>(L, M);
    return cudaGetLastError();
}

cudaError_t launch_regularize(const LbView &L, const MeshView &M, const RegParams &p, cudaStream_t s)
{
    k_regularize<<<1, 1024, 0, s>>>(L, M, p);
    return cudaGetLastError();
}

cudaError_t launch_observables(const LbView &L, const MeshView &M, cudaStream_t s)
{
    k_observables<<<1, 512, 0, s>>>(L, M);
    return cudaGetLastError();
}

cudaError_t launch_patch_from_mesh(const LbView &L, const MeshView &M, cudaStream_t s)
{
    k_patch<<<1, 256, 0, s>>>(L, M);
    return cudaGetLastError();
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
