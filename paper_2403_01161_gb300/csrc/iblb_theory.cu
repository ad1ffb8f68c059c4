// iblb_theory.cu -- the linear theory of Eq. (LT) (Sec. 2) along many
// velocity-gradient trajectories at once: each frame's strain held constant
// for `hold` time units (Sec. 3.2) and integrated with the classical
// fourth-order Runge-Kutta method in `substeps` steps per frame, FP64.  At
// each frame end S and the Sec. 2 observables of the droplet it describes
// are written.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "iblb_internal.h"
#include "iblb_device.cuh"

namespace iblb {
namespace {

// out[traj][frame][0..8]: S_xx, S_yy, S_zz, S_xy, S_xz, S_yz, lambda_max/R^2,
// beta (Eq. (beta), E of the frame; NaN when E = 0), D.
//
// Eq. (LT) on the deviation X = S - R^2 I is dX/dt = -a X + b E with a, b
// constant and E held over a frame, so one classical RK4 step of length h
// maps X to X* + P(z) (X - X*), X* = b E / a the frame's fixed point and
// P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = -a h, the method's stability
// polynomial (the four stages of RK4 applied to a linear constant-coefficient
// equation compose to exactly this affine map).  `substeps` steps of a frame
// are therefore X <- X* + P(z)^substeps (X - X*), the same RK4 result up to
// rounding order.  One thread per trajectory runs this recurrence over the
// frames and writes S; a second kernel, one thread per (trajectory, frame),
// takes the observables of every S in parallel.
__device__ __forceinline__ bool lt_params_ok(double tau, double R, double chi, double hold)
{
    return tau > 0.0 && R > 0.0 && chi >= 0.0 && hold > 0.0 && isfinite(tau) && isfinite(R) && isfinite(chi) &&
           isfinite(hold);
}

__global__ void __launch_bounds__(32) k_lt_recurrence(int n_traj, int n_frames, const double *__restrict__ A,
                                                       const double *__restrict__ params, int substeps,
                                                       double *__restrict__ out)
{
    const int tr = blockIdx.x * blockDim.x + threadIdx.x;
    if (tr >= n_traj) return;
    const double tau = params[4 * tr], R = params[4 * tr + 1], chi = params[4 * tr + 2], hold = params[4 * tr + 3];
    double *o = out + (size_t)tr * n_frames * 9;
    if (!lt_params_ok(tau, R, chi, hold)) {
        for (long long k = 0; k < 9LL * n_frames; ++k) o[k] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const double a = 40.0 * (chi + 1.0) / ((2.0 * chi + 3.0) * (19.0 * chi + 16.0)) / tau;
    const double b = 2.0 * R * R * 5.0 / (2.0 * chi + 3.0);
    const double z = -a * (hold / substeps);
    const double P = 1.0 + z * (1.0 + z * (0.5 + z * (1.0 / 6.0 + z * (1.0 / 24.0))));
    double Pn = 1.0, Pk = P;  // P^substeps by repeated squaring
    for (int e = substeps; e > 0; e >>= 1) {
        if (e & 1) Pn *= Pk;
        Pk *= Pk;
    }
    const double R2 = R * R, ba = b / a;
    double X[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // xx yy zz xy xz yz; a sphere at t = 0
    const double *Ak = A + (size_t)tr * n_frames * 9;
    for (int k = 0; k < n_frames; ++k, Ak += 9, o += 9) {
        const double E[6] = {Ak[0], Ak[4], Ak[8], 0.5 * (Ak[1] + Ak[3]), 0.5 * (Ak[2] + Ak[6]),
                             0.5 * (Ak[5] + Ak[7])};
        for (int c = 0; c < 6; ++c) {
            const double xs = ba * E[c];
            X[c] = xs + Pn * (X[c] - xs);
        }
        o[0] = R2 + X[0];
        o[1] = R2 + X[1];
        o[2] = R2 + X[2];
        o[3] = X[3];
        o[4] = X[4];
        o[5] = X[5];
    }
}

__global__ void __launch_bounds__(128) k_lt_observables(int n_traj, int n_frames, const double *__restrict__ A,
                                                        const double *__restrict__ params, double *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_traj * n_frames) return;
    const int tr = (int)(i / n_frames);
    const double tau = params[4 * tr], R = params[4 * tr + 1], chi = params[4 * tr + 2], hold = params[4 * tr + 3];
    if (!lt_params_ok(tau, R, chi, hold)) return;  // the row is NaN already
    double *o = out + 9 * i;
    const double *Ak = A + 9 * i;
    const double E[6] = {Ak[0], Ak[4], Ak[8], 0.5 * (Ak[1] + Ak[3]), 0.5 * (Ak[2] + Ak[6]), 0.5 * (Ak[5] + Ak[7])};
    double S[3][3] = {{o[0], o[3], o[4]}, {o[3], o[1], o[5]}, {o[4], o[5], o[2]}};
    double lam[3], v[3][3];
    jacobi3(S, lam, v);
    int imax = 0, imin = 0;
    for (int c = 1; c < 3; ++c) {
        if (lam[c] > lam[imax]) imax = c;
        if (lam[c] < lam[imin]) imin = c;
    }
    const double vx = v[0][imax], vy = v[1][imax], vz = v[2][imax];
    const double vEv = E[0] * vx * vx + E[1] * vy * vy + E[2] * vz * vz +
                       2.0 * (E[3] * vx * vy + E[4] * vx * vz + E[5] * vy * vz);
    const double nE = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + 2.0 * (E[3] * E[3] + E[4] * E[4] + E[5] * E[5]));
    const double p = sqrt(fmax(lam[imax], 0.0)), q = sqrt(fmax(lam[imin], 0.0));
    o[6] = lam[imax] / (R * R);
    o[7] = nE > 0.0 ? vEv / nE : __longlong_as_double(0x7ff8000000000000ll);
    o[8] = (p - q) / (p + q);
}

}  // namespace
}  // namespace iblb

extern "C" int ibl_linear_theory(int n_traj, int n_frames, const double *A, const double *params, int substeps,
                                 double *out, void *stream)
{
    if (n_traj < 1 || n_frames < 1) return iblb::iblb_set_error(IBL_EINVAL, "need at least one trajectory and frame");
    if (substeps < 1 || substeps > (1 << 20)) return iblb::iblb_set_error(IBL_EINVAL, "substeps must be in 1..2^20");
    if (!A || !params || !out) return iblb::iblb_set_error(IBL_EINVAL, "null device pointer");
    const long long cells = (long long)n_traj * n_frames;
    if (cells > 0x7fffffffLL * 128) return iblb::iblb_set_error(IBL_EINVAL, "too many trajectory frames");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    // small blocks spread the sequential recurrences over many SMs
    iblb::k_lt_recurrence<<<(unsigned)((n_traj + 31) / 32), 32, 0, s>>>(n_traj, n_frames, A, params, substeps, out);
    iblb::k_lt_observables<<<(unsigned)((cells + 127) / 128), 128, 0, s>>>(n_traj, n_frames, A, params, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return iblb::iblb_set_error(IBL_ECUDA, cudaGetErrorString(e));
    return IBL_OK;
}
