// iblb_device.cuh -- device helpers shared by the step kernels
// (iblb_kernels.cu) and the adjoint kernels (iblb_adjoint.cu): the D3Q19
// velocity set, compile-time loops, the Peskin 4-point stencil and its
// per-node broadcast, the surface-tension force of a triangle, block
// reductions and the 3x3 Jacobi eigen-solver.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
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

// Peskin 4-point stencil phi (Sec. 3.1), in the storage precision T.
template <typename T>
__device__ __forceinline__ T peskin_phi(T x)
{
    const T a = fabs(x);
    if (a < T(1)) return T(0.125) * (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a));
    if (a < T(2)) return T(0.125) * (T(5) - T(2) * a - sqrt(T(-7) + T(12) * a - T(4) * a * a));
    return T(0);
}

template <typename V>
__device__ __forceinline__ void cross3(const V a[3], const V b[3], V o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// The 4-point stencil along one axis starts at base = floor(r) - 1.  On a
// Zou-He axis all four nodes must be interior (1..n-2); periodic axes wrap.
struct AxisStencil {
    int base;
    bool ok;
};
__device__ __forceinline__ AxisStencil axis_stencil(double ra, int n, bool periodic)
{
    AxisStencil A;
    A.ok = fabs(ra) < 1e8;
    A.base = A.ok ? (int)floor(ra) - 1 : 0;
    if (A.ok && !periodic) A.ok = A.base >= 1 && A.base + 3 <= n - 2;
    return A;
}
__device__ __forceinline__ int wrap_index(int g, int n, bool periodic)
{
    if (periodic) {
        g %= n;
        if (g < 0) g += n;
    }
    return g;
}

constexpr int kLanesPerNode = 16;  // lane = (b, c) row of the 4x4x4 stencil
constexpr int kIbThreads = 128;    // threads per block of the node-group kernels
static_assert(kFwdNodesPerBlock * kFwdLanes == kIbThreads, "forward node-group blocks");

// Per-node stencil of the 16-lane group: lanes 0..2 compute, in FP64, the
// origin base_a = floor(r_a) - 1 and the exact fraction r_a - floor(r_a) of
// axis a, and every lane receives all three by shuffles.  The offset of
// stencil point k is then frac + (1 - k), the correctly rounded r - (base+k).
// L2 residency of the droplet-side working set.  Every step the outside
// lattice update streams the whole population array (about twice the L2 of
// a 128^3 box) through L2, which would evict the mesh arrays, the patch's
// populations and its force and velocity between two uses, so that each
// dependent access of the droplet chain would go to DRAM under full load.
// Accesses through an L2Keep carry an evict_last policy (PTX createpolicy
// and the .L2::cache_hint qualifier), which keeps those lines resident.
struct L2Keep {
    unsigned long long pol;
    __device__ __forceinline__ L2Keep() { asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol)); }
    __device__ __forceinline__ double ld(const double *a) const
    {
        double v;
        asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol) : "memory");
        return v;
    }
    __device__ __forceinline__ float ld(const float *a) const
    {
        float v;
        asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol) : "memory");
        return v;
    }
    __device__ __forceinline__ int ld(const int *a) const
    {
        int v;
        asm volatile("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol) : "memory");
        return v;
    }
    __device__ __forceinline__ void st(double *a, double v) const
    {
        asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
    }
    __device__ __forceinline__ void st(float *a, float v) const
    {
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
    }
    __device__ __forceinline__ void red_add(float *a, float v) const
    {
        asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
    }
    __device__ __forceinline__ void red_add(double *a, double v) const
    {
        asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
    }
    // three components of a 4-wide node record (16-byte aligned for float,
    // 32-byte for double): one vector access per record in FP32
    __device__ __forceinline__ void ld3(const float *a, float &x, float &y, float &z) const
    {
        float w;
        asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(x), "=f"(y), "=f"(z), "=f"(w)
                     : "l"(a), "l"(pol)
                     : "memory");
    }
    __device__ __forceinline__ void ld3(const double *a, double &x, double &y, double &z) const
    {
        asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(x), "=d"(y) : "l"(a), "l"(pol) : "memory");
        z = ld(a + 2);
    }
    __device__ __forceinline__ void st3(float *a, float x, float y, float z) const
    {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(x), "f"(y), "f"(z),
                     "f"(0.f), "l"(pol)
                     : "memory");
    }
    __device__ __forceinline__ void st3(double *a, double x, double y, double z) const
    {
        asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(a), "d"(x), "d"(y), "l"(pol) : "memory");
        st(a + 2, z);
    }
    __device__ __forceinline__ void red_add3(float *a, float x, float y, float z) const
    {
        asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(x), "f"(y),
                     "f"(z), "f"(0.f), "l"(pol)
                     : "memory");
    }
    __device__ __forceinline__ void red_add3(double *a, double x, double y, double z) const
    {
        red_add(a, x);
        red_add(a + 1, y);
        red_add(a + 2, z);
    }
};

// Plain-policy access to the three components of a 4-wide node record.
__device__ __forceinline__ void rec_ld3(const float *a, float &x, float &y, float &z)
{
    const float4 v = *reinterpret_cast<const float4 *>(a);
    x = v.x;
    y = v.y;
    z = v.z;
}
__device__ __forceinline__ void rec_ld3(const double *a, double &x, double &y, double &z)
{
    const double2 v = *reinterpret_cast<const double2 *>(a);
    x = v.x;
    y = v.y;
    z = a[2];
}
__device__ __forceinline__ void rec_st3(float *a, float x, float y, float z)
{
    *reinterpret_cast<float4 *>(a) = make_float4(x, y, z, 0.f);
}
__device__ __forceinline__ void rec_st3(double *a, double x, double y, double z)
{
    *reinterpret_cast<double2 *>(a) = make_double2(x, y);
    a[2] = z;
}
__device__ __forceinline__ void rec_red3(float *a, float x, float y, float z)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(x), "f"(y), "f"(z), "f"(0.f) : "memory");
}
__device__ __forceinline__ void rec_red3(double *a, double x, double y, double z)
{
    atomicAdd(a, x);
    atomicAdd(a + 1, y);
    atomicAdd(a + 2, z);
}

// The same interface with the default policy (plain loads, stores and
// reductions), for the batched ensemble kernels: the droplet-side working
// set of many members together exceeds L2, where lines kept with evict_last
// would only displace the lattice update's reuse.
struct L2Plain {
    template <class V>
    __device__ __forceinline__ V ld(const V *a) const
    {
        return *a;
    }
    template <class V>
    __device__ __forceinline__ void st(V *a, V v) const
    {
        *a = v;
    }
    __device__ __forceinline__ void red_add(float *a, float v) const { atomicAdd(a, v); }
    __device__ __forceinline__ void red_add(double *a, double v) const { atomicAdd(a, v); }
    template <class V>
    __device__ __forceinline__ void ld3(const V *a, V &x, V &y, V &z) const
    {
        rec_ld3(a, x, y, z);
    }
    template <class V>
    __device__ __forceinline__ void st3(V *a, V x, V y, V z) const
    {
        rec_st3(a, x, y, z);
    }
    template <class V>
    __device__ __forceinline__ void red_add3(V *a, V x, V y, V z) const
    {
        rec_red3(a, x, y, z);
    }
};

struct NodeStencil {
    int base[3];
    double frac[3];
    bool ok;
};
template <int LANES = kLanesPerNode, class P = L2Keep>
__device__ __forceinline__ NodeStencil node_stencil(const LbView &L, const double *r, int lane,
                                                    const P *keep = nullptr)
{
    double ra = 0.0, fr = 0.0;
    int base = 0;
    bool ok = true;
    if (lane < 3) {
        ra = keep ? keep->ld(r + lane) : r[lane];
        // select by value: indexing the parameter arrays with a runtime lane
        // would copy the kernel parameters to local memory
        const int na = lane == 0 ? L.n[0] : (lane == 1 ? L.n[1] : L.n[2]);
        const int bca = lane == 0 ? L.bc[0] : (lane == 1 ? L.bc[1] : L.bc[2]);
        const AxisStencil A = axis_stencil(ra, na, bca == IBL_BC_PERIODIC);
        ok = A.ok;
        base = A.base;
        fr = ok ? ra - floor(ra) : 0.0;
    }
    const int w0 = (threadIdx.x & 31) & ~(LANES - 1);
    NodeStencil S;
    S.ok = true;
    // every lane executes every full-mask shuffle (no short-circuit around
    // them: a lane that skipped one would leave the others waiting)
    for (int a = 0; a < 3; ++a) {
        S.base[a] = __shfl_sync(0xffffffffu, base, w0 + a);
        S.frac[a] = __shfl_sync(0xffffffffu, fr, w0 + a);
        const int ok_a = __shfl_sync(0xffffffffu, ok ? 1 : 0, w0 + a);
        S.ok = S.ok && (ok_a != 0);
    }
    return S;
}

// Weights of the lane's x-row (w[0..3]) and of its y and z rows, in the
// storage precision: offsets frac + (1 - k); in FP32 the fraction is
// rounded to float first, in FP64 the offsets are the correctly rounded
// r - (base + k).
template <typename T>
__device__ __forceinline__ void stencil_weights(const NodeStencil &S, int b, int c, T w[4], T &wy, T &wz)
{
    if constexpr (sizeof(T) == 8) {
        for (int a = 0; a < 4; ++a) w[a] = peskin_phi<T>(S.frac[0] + (double)(1 - a));
        wy = peskin_phi<T>(S.frac[1] + (double)(1 - b));
        wz = peskin_phi<T>(S.frac[2] + (double)(1 - c));
    } else {
        const T fx = T(S.frac[0]), fy = T(S.frac[1]), fz = T(S.frac[2]);
        for (int a = 0; a < 4; ++a) w[a] = peskin_phi<T>(fx + T(1 - a));
        wy = peskin_phi<T>(fy + T(1 - b));
        wz = peskin_phi<T>(fz + T(1 - c));
    }
}

// Whether lattice node (x, y, z) lies in the droplet patch stored in buffer
// `buf` of control block c (periodic axes wrap).
__device__ __forceinline__ bool node_in_patch(const LbView &L, const Ctl *c, int buf, int x, int y, int z)
{
    int dx = x - c->patch_lo[buf][0], dy = y - c->patch_lo[buf][1], dz = z - c->patch_lo[buf][2];
    if (L.bc[0] == IBL_BC_PERIODIC && dx < 0) dx += L.n[0];
    if (L.bc[1] == IBL_BC_PERIODIC && dy < 0) dy += L.n[1];
    if (L.bc[2] == IBL_BC_PERIODIC && dz < 0) dz += L.n[2];
    // an empty patch has extent -1: no node is inside
    return c->patch_ext[buf][0] >= 0 && (unsigned)dx <= (unsigned)c->patch_ext[buf][0] &&
           (unsigned)dy <= (unsigned)c->patch_ext[buf][1] && (unsigned)dz <= (unsigned)c->patch_ext[buf][2];
}

// Surface-tension force of triangle t on its vertex in position `slot`
// (Eq. (pi_drop), F_i = -sigma dA/dx_i summed over the triangles around i):
// m_t x (x_{slot+2} - x_{slot+1}) with the scaled unit normal
// m_t = -sigma/2 N/|N|, N = (x1 - x0) x (x2 - x0).  Positions are FP64; the
// edge vectors are formed in FP64 and the rest runs in G (the step uses
// FP64 mesh geometry for either population precision).
template <typename G>
__device__ __forceinline__ void tri_force(const MeshView &M, const int t, const int slot, G g[3])
{
    double x[3][3];
    for (int k = 0; k < 3; ++k) {
        const int v = M.tris[3 * t + k];
        for (int a = 0; a < 3; ++a) x[k][a] = M.r[3 * v + a];
    }
    G e1[3], e2[3], N[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = G(x[1][a] - x[0][a]);
        e2[a] = G(x[2][a] - x[0][a]);
    }
    cross3(e1, e2, N);
    const G s = G(-0.5) * G(M.sigma) * rsqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    const G m[3] = {s * N[0], s * N[1], s * N[2]};
    const int kp = slot == 2 ? 0 : slot + 1, km = slot == 0 ? 2 : slot - 1;
    const G dd[3] = {G(x[km][0] - x[kp][0]), G(x[km][1] - x[kp][1]), G(x[km][2] - x[kp][2])};
    cross3(m, dd, g);
}

// The same force in two stages, so that the FP64 normal of each triangle is
// evaluated once per step instead of once per corner: tri_moment gives m_t
// = -sigma N_t / (2 |N_t|) (the m of tri_force<double>, bit for bit), and
// tri_force_m the force on corner `slot` from a stored m_t.
template <class P>
__device__ __forceinline__ void tri_moment(const MeshView &M, const int t, double m[3], const P &K)
{
    double x[3][3];
    for (int k = 0; k < 3; ++k) {
        const int v = K.ld(M.tris + 3 * t + k);
        for (int a = 0; a < 3; ++a) x[k][a] = K.ld(M.r + 3 * v + a);
    }
    double e1[3], e2[3], N[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = x[1][a] - x[0][a];
        e2[a] = x[2][a] - x[0][a];
    }
    cross3(e1, e2, N);
    const double s = -0.5 * M.sigma * rsqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    for (int a = 0; a < 3; ++a) m[a] = s * N[a];
}

template <class P>
__device__ __forceinline__ void tri_force_m(const MeshView &M, const int t, const int slot, const double m[3],
                                            double g[3], const P &K)
{
    const int kp = slot == 2 ? 0 : slot + 1, km = slot == 0 ? 2 : slot - 1;
    const int vp = K.ld(M.tris + 3 * t + kp), vm = K.ld(M.tris + 3 * t + km);
    double dd[3];
    for (int a = 0; a < 3; ++a) dd[a] = K.ld(M.r + 3 * vm + a) - K.ld(M.r + 3 * vp + a);
    cross3(m, dd, g);
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


}  // namespace

// Launch with an explicit scheduling priority (0 = the stream's own).  The
// attribute is recorded into the kernel node under stream capture, which the
// stream priority alone is not.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_p(void (*k)(KArgs...), dim3 g, dim3 b, cudaStream_t s, int prio, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = prio != 0 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// ---- bulk asynchronous copies into shared memory (sm_90 and later) -------
// A bulk copy (cp.async.bulk) moves a contiguous run of global memory into
// shared memory without occupying registers and signals completion on an
// mbarrier in shared memory by the bytes it delivered (complete_tx).  Both
// addresses and the size must be multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisations visible to the asynchronous proxy (the copy
// engine) before any copy signals them.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of copies to be completed in the
// barrier's current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the phase with parity `parity` of the barrier has completed;
// gives up after `limit_ns` nanoseconds of the global timer and returns
// false then.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned long long limit_ns)
{
    const unsigned a = smem_addr(bar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

}  // namespace iblb
