// iblb_theory.cu -- the linear theory of Eq. (LT) (Sec. 2) along many
// velocity-gradient trajectories at once: one thread per trajectory, each
// frame's strain held constant for `hold` time units (Sec. 3.2) and
// integrated with the classical fourth-order Runge-Kutta method in
// `substeps` steps per frame, FP64.  At each frame end the thread writes S
// and the Sec. 2 observables of the droplet it describes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "iblb_internal.h"
#include "iblb_device.cuh"

namespace iblb {
namespace {

// out[traj][frame][0..8]: S_xx, S_yy, S_zz, S_xy, S_xz, S_yz, lambda_max/R^2,
// beta (Eq. (beta), E of the frame; NaN when E = 0), D.
__global__ void __launch_bounds__(32) k_linear_theory(int n_traj, int n_frames, const double *__restrict__ A,
                                                      const double *__restrict__ params, int substeps,
                                                      double *__restrict__ out)
{
    const int tr = blockIdx.x * blockDim.x + threadIdx.x;
    if (tr >= n_traj) return;
    const double tau = params[4 * tr], R = params[4 * tr + 1], chi = params[4 * tr + 2], hold = params[4 * tr + 3];
    double *o = out + (size_t)tr * n_frames * 9;
    const bool ok = tau > 0.0 && R > 0.0 && chi >= 0.0 && hold > 0.0 && isfinite(tau) && isfinite(R) &&
                    isfinite(chi) && isfinite(hold);
    if (!ok) {
        for (long long k = 0; k < 9LL * n_frames; ++k) o[k] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    // Eq. (LT) on the deviation X = S - R^2 I:  dX/dt = -a X + b E
    const double a = 40.0 * (chi + 1.0) / ((2.0 * chi + 3.0) * (19.0 * chi + 16.0)) / tau;
    const double b = 2.0 * R * R * 5.0 / (2.0 * chi + 3.0);
    const double h = hold / substeps;
    double X[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // xx yy zz xy xz yz; a sphere at t = 0
    const double *Ak = A + (size_t)tr * n_frames * 9;
    for (int k = 0; k < n_frames; ++k, Ak += 9, o += 9) {
        const double E[6] = {Ak[0], Ak[4], Ak[8], 0.5 * (Ak[1] + Ak[3]), 0.5 * (Ak[2] + Ak[6]),
                             0.5 * (Ak[5] + Ak[7])};
        double bE[6];
        for (int c = 0; c < 6; ++c) bE[c] = b * E[c];
        for (int s = 0; s < substeps; ++s) {
            double k1[6], k2[6], k3[6], k4[6], y[6];
            for (int c = 0; c < 6; ++c) k1[c] = bE[c] - a * X[c];
            for (int c = 0; c < 6; ++c) y[c] = X[c] + 0.5 * h * k1[c];
            for (int c = 0; c < 6; ++c) k2[c] = bE[c] - a * y[c];
            for (int c = 0; c < 6; ++c) y[c] = X[c] + 0.5 * h * k2[c];
            for (int c = 0; c < 6; ++c) k3[c] = bE[c] - a * y[c];
            for (int c = 0; c < 6; ++c) y[c] = X[c] + h * k3[c];
            for (int c = 0; c < 6; ++c) k4[c] = bE[c] - a * y[c];
            for (int c = 0; c < 6; ++c) X[c] += h / 6.0 * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
        }
        const double R2 = R * R;
        double S[3][3] = {{R2 + X[0], X[3], X[4]}, {X[3], R2 + X[1], X[5]}, {X[4], X[5], R2 + X[2]}};
        for (int c = 0; c < 3; ++c) o[c] = S[c][c];
        o[3] = X[3];
        o[4] = X[4];
        o[5] = X[5];
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
        const double nE = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2] +
                               2.0 * (E[3] * E[3] + E[4] * E[4] + E[5] * E[5]));
        const double p = sqrt(fmax(lam[imax], 0.0)), q = sqrt(fmax(lam[imin], 0.0));
        o[6] = lam[imax] / R2;
        o[7] = nE > 0.0 ? vEv / nE : __longlong_as_double(0x7ff8000000000000ll);
        o[8] = (p - q) / (p + q);
    }
}

}  // namespace
}  // namespace iblb

extern "C" int ibl_linear_theory(int n_traj, int n_frames, const double *A, const double *params, int substeps,
                                 double *out, void *stream)
{
    if (n_traj < 1 || n_frames < 1) return iblb::iblb_set_error(IBL_EINVAL, "need at least one trajectory and frame");
    if (substeps < 1 || substeps > (1 << 20)) return iblb::iblb_set_error(IBL_EINVAL, "substeps must be in 1..2^20");
    if (!A || !params || !out) return iblb::iblb_set_error(IBL_EINVAL, "null device pointer");
    const unsigned blocks = (unsigned)((n_traj + 31) / 32);
    iblb::k_linear_theory<<<blocks, 32, 0, static_cast<cudaStream_t>(stream)>>>(n_traj, n_frames, A, params,
                                                                               substeps, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return iblb::iblb_set_error(IBL_ECUDA, cudaGetErrorString(e));
    return IBL_OK;
}
