/*
 * iblb_oracle.c -- plain FP64 CPU oracle of one immersed-boundary lattice
 * Boltzmann (IBLB) droplet time step, written from Taglienti, Guglietta and
 * Sbragaglia, "Droplet dynamics in homogeneous isotropic turbulence with the
 * immersed boundary-lattice Boltzmann method" (arXiv:2403.01161).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load this
 * library: only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no source, header, table or helper with the
 * CUDA path.  Every loop is serial and in the order the method states,
 * except the lattice collide/stream loop, which is split over z-planes with
 * OpenMP (each node is independent there, so the result does not depend on
 * the thread count).
 *
 * What each function follows (paper section / equation):
 *   D3Q19 weights ............ Sec. 3.1, weights listed after Eq. (equilibriumLB)
 *   equilibrium .............. Eq. (equilibriumLB), read with -u.u/(2 cs^2)
 *   Guo source ............... Sec. 3.1, Guo forcing term S_i
 *   moments .................. Eq. (density_velocity_LB), half-force momentum
 *   BGK + streaming .......... Eq. (LBMEQ), Eq. (collision)
 *   face Zou-He rule ......... Eq. (ZH_bulk) and its bounce-back limit Eq. (standard BB)
 *   edge rule ................ Eq. (ZH_edges) + buried links Eq. (zh-buried-links-edges)
 *   corner rule .............. Eq. (zh-buried-links-corners)
 *   wall velocity ............ Eq. (velo_facce_cubo_da_gradiente); optionally
 *                              centred on the droplet's centre of mass (Sec. 3.2)
 *   Peskin 4-point kernel .... Sec. 3.1, phi(x) after Eq. (ibm_force_d)
 *   spread / interpolate ..... Eq. (ibm_force_d) (a) and (b)
 *   advection ................ Eq. (fwd_euler)
 *   nodal forces ............. Eq. (pi_drop): F_i = -sigma dA/dx_i
 *   regularisation ........... Sec. 3.3, Eqs. (extended laplacian smoothing),
 *                              (HC_algo_full), (distanceregularization)
 *   frame schedule ........... Sec. 3.2, the four-step trajectory loop
 *   viscosity ratio chi ...... Sec. 2 (droplet viscosity chi mu): tau inside the
 *                              droplet from an even-odd ray count over the mesh
 *
 * Parity status: every function is pinned by tests/test_oracle_*.py against
 * closed forms, invariants or brute force (the re-centred face velocity
 * against the pinned volume centroid, the ray indicator against the
 * half-space test and the solid-angle winding number; interpolation and
 * advection by exact transport in a uniform flow, exact reproduction of a
 * linear velocity field and the (k - 1/2) g velocity of a fluid under a
 * uniform force).  The edge and corner rules with a moving wall
 * (EDGE_COUNTER_SLIP) are a reading of Eqs. (ZH_edges),
 * (zh-buried-links-edges) and (zh-buried-links-corners), pinned by what that
 * reading is built to meet: the rest state, the no-slip of an edge at rest,
 * the exact wall momentum of every edge and corner node for any input, and
 * a linear shear kept inside the box.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 velocities, the oracle's own order: rest, six axis links, twelve
 * face diagonals.  Sec. 3.1: c_0 is the rest population. */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static const double CS2 = 1.0 / 3.0; /* c_s^2, Sec. 3.1 after Eq. (tau_to_nu) */

/* w_i = w(|c_i|^2): 1/3, 1/18, 1/36 (Sec. 3.1). */
static double weight(int i)
{
    int c2 = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
    if (c2 == 0) return 1.0 / 3.0;
    if (c2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* index of -c_i, found by search */
static int opposite(int i)
{
    for (int j = 0; j < Q; ++j)
        if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) return j;
    return -1;
}

static double cdot(int i, const double v[3])
{
    return CV[i][0] * v[0] + CV[i][1] * v[1] + CV[i][2] * v[2];
}

int orc_velocity(int i, int out[3])
{
    if (i < 0 || i >= Q) return -1;
    out[0] = CV[i][0]; out[1] = CV[i][1]; out[2] = CV[i][2];
    return 0;
}

double orc_weight(int i) { return (i >= 0 && i < Q) ? weight(i) : 0.0; }

/* Eq. (equilibriumLB) with the quadratic term read as -u.u/(2 c_s^2). */
void orc_equilibrium(double rho, const double u[3], double feq[Q])
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = cdot(i, u);
        feq[i] = weight(i) * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Guo source, Sec. 3.1:
 *   S_i = (1 - 1/(2 tau)) (w_i / c_s^2) [ ((c_i.u)/c_s^2 + 1) c_i - u ] . F */
void orc_guo_source(double tau, const double u[3], const double F[3], double S[Q])
{
    double pre = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < Q; ++i) {
        double cu = cdot(i, u);
        double v[3];
        for (int a = 0; a < 3; ++a) v[a] = (cu / CS2 + 1.0) * CV[i][a] - u[a];
        S[i] = pre * weight(i) / CS2 * (v[0] * F[0] + v[1] * F[1] + v[2] * F[2]);
    }
}

/* Peskin 4-point stencil phi(x), Sec. 3.1. */
double orc_peskin_phi(double x)
{
    double a = fabs(x);
    if (a < 1.0) return 0.125 * (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a));
    if (a < 2.0) return 0.125 * (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
    return 0.0;
}

/* ---------------------------------------------------------------------------
 * Box boundary.  side[a] = -1 on the face l_a = 0, +1 on the face l_a = L_a,
 * 0 otherwise (or on a periodic axis).  A population f_j is unknown after
 * streaming when the node it would come from, x - c_j, lies outside the box:
 * c_ja * side[a] < 0 on some boundary axis.
 * ------------------------------------------------------------------------- */
enum { EDGE_COUNTER_SLIP = 0, EDGE_PAPER_LITERAL = 1 };

static int unknown(int j, const int side[3])
{
    for (int a = 0; a < 3; ++a)
        if (side[a] != 0 && CV[j][a] * side[a] < 0) return 1;
    return 0;
}

/* Face node, case (a): Eq. (ZH_bulk), with the Zou-He closure for rho
 * rho = (sum_{c.n=0} f + 2 sum_{c.n_out>0} f) / (1 + u_w.n_out). */
static double bc_face(double f[Q], int a, int s, const double uw[3])
{
    double n[3] = {0, 0, 0};
    n[a] = (double)s; /* outward normal; the rule does not depend on its sign */
    double sum_tan = 0.0, sum_out = 0.0;
    for (int k = 0; k < Q; ++k) {
        if (CV[k][a] == 0) sum_tan += f[k];
        else if (CV[k][a] * s > 0) sum_out += f[k];
    }
    double rho = (sum_tan + 2.0 * sum_out) / (1.0 + uw[a] * s);
    double g[Q];
    memcpy(g, f, sizeof g);
    for (int j = 0; j < Q; ++j) {
        if (!(CV[j][a] * s < 0)) continue;
        int i = opposite(j); /* c_i points out of the box; f_i is known */
        double t[3] = {(double)CV[i][0], (double)CV[i][1], (double)CV[i][2]};
        double cn = t[0] * n[0] + t[1] * n[1] + t[2] * n[2];
        for (int b = 0; b < 3; ++b) t[b] -= cn * n[b];
        double tnorm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        double corr = 0.0;
        for (int k = 0; k < Q; ++k) {
            double ck_n = fabs(CV[k][0] * n[0] + CV[k][1] * n[1] + CV[k][2] * n[2]);
            double tc = t[0] * CV[k][0] + t[1] * CV[k][1] + t[2] * CV[k][2];
            corr += f[k] * tc * (1.0 - ck_n);
        }
        double tu = t[0] * uw[0] + t[1] * uw[1] + t[2] * uw[2];
        g[j] = f[i] - (2.0 - tnorm) * rho / 6.0 * cdot(i, uw) - rho / 3.0 * tu + 0.5 * corr;
    }
    memcpy(f, g, sizeof g);
    return rho;
}

/* Edge node, case (b): Eq. (ZH_edges) for the non-buried unknowns, t_i read
 * as c_i projected on the edge line, then the buried links of
 * Eq. (zh-buried-links-edges) and f_0 = 12 f^(1,2).
 *
 * EDGE_PAPER_LITERAL takes the equation as printed: the tangential sum with
 * a minus sign and no wall velocity.  Read with the face rule's convention
 * (c_i outgoing, f_{-i} reflected), that sign adds the along-edge momentum
 * of the edge-line pair a second time instead of removing it, so an edge at
 * rest slips.  EDGE_COUNTER_SLIP is the face rule's construction carried to
 * two normals, rho0 = 1:
 *   f_{-i} = f_i - 2 w_i rho0 (c_i.u_w)/c_s^2 - rho0/12 (t_i.u_w)
 *            + 1/4 sum_j f_j (t_i.c_j)(1 - |c_j.n1|)(1 - |c_j.n2|),
 * whose sum cancels the edge-line momentum (four reflected links with a
 * component along the edge, 1/4 each) and whose t_i.u_w term restores the
 * wall's own share of it (the edge-line pair carries 1/3 of rho u in
 * equilibrium, 1/4 of which each link would remove); and each buried link
 * gets f^(1,2) plus its half of the moving-wall difference,
 * w_j rho0 (c_j.u_w)/c_s^2.  The node then carries the momentum rho0 u_w
 * exactly, whatever arrived, and an edge at rest imposes no slip. */
static void bc_edge(double f[Q], const int side[3], const double uw[3], int rule)
{
    double n1[3] = {0, 0, 0}, n2[3] = {0, 0, 0};
    int got = 0;
    for (int a = 0; a < 3; ++a) {
        if (side[a] == 0) continue;
        if (got == 0) n1[a] = -side[a]; else n2[a] = -side[a]; /* inward normals */
        ++got;
    }
    double g[Q];
    memcpy(g, f, sizeof g);
    for (int j = 1; j < Q; ++j) {
        if (!unknown(j, side)) continue;
        int i = opposite(j);
        if (unknown(i, side)) continue; /* buried link, set below */
        double c1 = CV[i][0] * n1[0] + CV[i][1] * n1[1] + CV[i][2] * n1[2];
        double c2 = CV[i][0] * n2[0] + CV[i][1] * n2[1] + CV[i][2] * n2[2];
        double t[3];
        for (int b = 0; b < 3; ++b) t[b] = CV[i][b] - c1 * n1[b] - c2 * n2[b];
        double corr = 0.0;
        for (int k = 0; k < Q; ++k) {
            double k1 = fabs(CV[k][0] * n1[0] + CV[k][1] * n1[1] + CV[k][2] * n1[2]);
            double k2 = fabs(CV[k][0] * n2[0] + CV[k][1] * n2[1] + CV[k][2] * n2[2]);
            double tc = t[0] * CV[k][0] + t[1] * CV[k][1] + t[2] * CV[k][2];
            corr += f[k] * tc * (1.0 - k1) * (1.0 - k2);
        }
        double v;
        if (rule == EDGE_PAPER_LITERAL) {
            v = f[i] - 0.25 * corr;
        } else {
            double tu = t[0] * uw[0] + t[1] * uw[1] + t[2] * uw[2];
            v = f[i] - 2.0 * weight(i) * 1.0 * cdot(i, uw) / CS2 - 1.0 / 12.0 * tu + 0.25 * corr;
        }
        g[j] = v;
    }
    double e[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2],
                   n1[0] * n2[1] - n1[1] * n2[0]};
    double s[3] = {n1[0] + n2[0], n1[1] + n2[1], n1[2] + n2[2]};
    double fb = 0.0;
    for (int i = 1; i < Q; ++i) {
        double c2 = (double)(CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2]);
        double ce = fabs(CV[i][0] * e[0] + CV[i][1] * e[1] + CV[i][2] * e[2]);
        double cs = fabs(CV[i][0] * s[0] + CV[i][1] * s[1] + CV[i][2] * s[2]) / c2;
        double wgt = 1.0 - (1.0 - ce) * (1.0 - cs);
        if (wgt != 0.0) fb += g[i] * wgt; /* buried terms have weight 0 */
    }
    fb /= 22.0;
    for (int j = 1; j < Q; ++j) {
        if (!(unknown(j, side) && unknown(opposite(j), side))) continue;
        g[j] = fb;
        if (rule == EDGE_COUNTER_SLIP) g[j] += weight(j) * 1.0 * cdot(j, uw) / CS2;
    }
    g[0] = 12.0 * fb;
    memcpy(f, g, sizeof g);
}

/* Corner node, case (c): Eq. (zh-buried-links-corners) and f_0 = 12 f^(1..6).
 * The paper gives no rule for the non-buried unknowns (three normals leave
 * no tangential direction); they take moving-wall bounce-back, and under
 * EDGE_COUNTER_SLIP each buried link adds its half of the moving-wall
 * difference, w_j rho0 (c_j.u_w)/c_s^2, as at an edge, so that the node
 * carries rho0 u_w exactly.  EDGE_PAPER_LITERAL: plain bounce-back and the
 * buried value alone. */
static void bc_corner(double f[Q], const int side[3], const double uw[3], int rule)
{
    double s[3] = {(double)-side[0], (double)-side[1], (double)-side[2]}; /* n1+n2+n3 */
    double g[Q];
    memcpy(g, f, sizeof g);
    for (int j = 1; j < Q; ++j) {
        if (!unknown(j, side)) continue;
        double cs = CV[j][0] * s[0] + CV[j][1] * s[1] + CV[j][2] * s[2];
        if (cs == 0.0) continue; /* buried */
        int i = opposite(j);
        double v = f[i];
        if (rule == EDGE_COUNTER_SLIP) v -= 2.0 * weight(i) * 1.0 * cdot(i, uw) / CS2;
        g[j] = v;
    }
    double fb = 0.0;
    for (int i = 1; i < Q; ++i) {
        double c2 = (double)(CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2]);
        double wgt = fabs(CV[i][0] * s[0] + CV[i][1] * s[1] + CV[i][2] * s[2]) / c2;
        if (wgt != 0.0) fb += g[i] * wgt;
    }
    fb /= 18.0;
    for (int j = 1; j < Q; ++j) {
        double cs = CV[j][0] * s[0] + CV[j][1] * s[1] + CV[j][2] * s[2];
        if (cs != 0.0) continue;
        g[j] = fb;
        if (rule == EDGE_COUNTER_SLIP) g[j] += weight(j) * 1.0 * cdot(j, uw) / CS2;
    }
    g[0] = 12.0 * fb;
    memcpy(f, g, sizeof g);
}

/* Reconstructs the unknown populations of one boundary node in place. */
int orc_bc_node(double f[Q], const int side[3], const double uw[3], int rule)
{
    int nb = (side[0] != 0) + (side[1] != 0) + (side[2] != 0);
    if (nb == 1) {
        for (int a = 0; a < 3; ++a)
            if (side[a] != 0) bc_face(f, a, side[a], uw);
    } else if (nb == 2) {
        bc_edge(f, side, uw, rule);
    } else if (nb == 3) {
        bc_corner(f, side, uw, rule);
    }
    return nb;
}

/* ---------------------------------------------------------------------------
 * Surface tension nodal forces, Eq. (pi_drop): with Pi = sigma I_2 the force
 * on node i is -sigma dA/dx_i.  For a triangle (a,b,c), counter-clockwise
 * about its outward unit normal n, dA/da = 1/2 n x (c - b), cyclically.
 * ------------------------------------------------------------------------- */
static void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_nodal_forces(int nv, const double *r, int nt, const int *tri, double sigma, double *F)
{
    memset(F, 0, sizeof(double) * 3 * (size_t)nv);
    for (int t = 0; t < nt; ++t) {
        const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        const double *x0 = r + 3 * v[0], *x1 = r + 3 * v[1], *x2 = r + 3 * v[2];
        double e1[3], e2[3], N[3];
        for (int a = 0; a < 3; ++a) { e1[a] = x1[a] - x0[a]; e2[a] = x2[a] - x0[a]; }
        cross(e1, e2, N);
        double len = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        double n[3] = {N[0] / len, N[1] / len, N[2] / len};
        for (int k = 0; k < 3; ++k) {
            const double *xp = r + 3 * v[(k + 1) % 3], *xm = r + 3 * v[(k + 2) % 3];
            double d[3] = {xm[0] - xp[0], xm[1] - xp[1], xm[2] - xp[2]};
            double g[3];
            cross(n, d, g);
            for (int a = 0; a < 3; ++a) F[3 * v[k] + a] += -sigma * 0.5 * g[a];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Enclosed volume and volume centroid of a closed, outward-oriented triangle
 * mesh, summed over the signed tetrahedra (x_0, a, b, c) of its triangles;
 * each tetrahedron's centroid is the mean of its four corners.
 */
void orc_enclosed_volume(int nv, const double *x, int nt, const int *tri, double *V, double *c)
{
    (void)nv;
    double v = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < nt; ++t) {
        double p[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) p[k][a] = x[3 * tri[3 * t + k] + a] - x[a];
        double bc[3];
        cross(p[1], p[2], bc);
        double vt = (p[0][0] * bc[0] + p[0][1] * bc[1] + p[0][2] * bc[2]) / 6.0;
        v += vt;
        for (int a = 0; a < 3; ++a) m[a] += vt * (p[0][a] + p[1][a] + p[2][a]) / 4.0;
    }
    *V = v;
    for (int a = 0; a < 3; ++a) c[a] = x[a] + m[a] / v;
}

/* Scales the mesh about its volume centroid so that it encloses V_target. */
void orc_restore_volume(int nv, double *x, int nt, const int *tri, double V_target)
{
    double V, c[3];
    orc_enclosed_volume(nv, x, nt, tri, &V, c);
    double f = cbrt(V_target / V);
    for (int i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) x[3 * i + a] = c[a] + f * (x[3 * i + a] - c[a]);
}

/* ---------------------------------------------------------------------------
 * Mesh regularisation, Sec. 3.3 (extended Laplacian smoothing).
 * plus_sign = 1 reads the correction of Eq. (HC_algo_full) as
 *   x_p <- x_p - (gamma b_i + (1-gamma)/N_i sum_j b_j)
 * plus_sign = 0 uses the sign as printed, -(1-gamma)/N_i sum_j b_j.
 * Returns the number of iterations; *converged = 1 if the exit test held.
 * ------------------------------------------------------------------------- */
int orc_regularize(int nv, double *x, const int *nb_ptr, const int *nb_idx, double alpha,
                   double gamma, double tol, int max_iter, int plus_sign, int *converged)
{
    size_t sz = sizeof(double) * 3 * (size_t)nv;
    double *xo = (double *)malloc(sz), *xp = (double *)malloc(sz);
    double *xq = (double *)malloc(sz), *xb = (double *)malloc(sz);
    memcpy(xo, x, sz);
    memcpy(xp, x, sz);
    int it = 0, ok = 0;
    while (it < max_iter) {
        ++it;
        memcpy(xq, xp, sz); /* step 1 */
        for (int i = 0; i < nv; ++i) { /* step 2 */
            int ni = nb_ptr[i + 1] - nb_ptr[i];
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = nb_ptr[i]; k < nb_ptr[i + 1]; ++k) s += xq[3 * nb_idx[k] + a];
                xp[3 * i + a] = alpha * xo[3 * i + a] + (1.0 - alpha) / ni * s;
            }
        }
        for (int i = 0; i < nv; ++i) /* Eq. (distanceregularization) */
            for (int a = 0; a < 3; ++a)
                xb[3 * i + a] = xp[3 * i + a] - (alpha * xo[3 * i + a] + (1.0 - alpha) * xq[3 * i + a]);
        double sg = plus_sign ? 1.0 : -1.0;
        for (int i = 0; i < nv; ++i) { /* step 3, Eq. (HC_algo_full) */
            int ni = nb_ptr[i + 1] - nb_ptr[i];
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int k = nb_ptr[i]; k < nb_ptr[i + 1]; ++k) s += xb[3 * nb_idx[k] + a];
                xp[3 * i + a] -= gamma * xb[3 * i + a] + sg * (1.0 - gamma) / ni * s;
            }
        }
        double maxd = 0.0; /* step 4 */
        for (int i = 0; i < nv; ++i) {
            double d0 = xp[3 * i] - xq[3 * i], d1 = xp[3 * i + 1] - xq[3 * i + 1],
                   d2 = xp[3 * i + 2] - xq[3 * i + 2];
            double d = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            if (d > maxd) maxd = d;
        }
        if (maxd < tol) { ok = 1; break; }
    }
    memcpy(x, xp, sz);
    free(xo); free(xp); free(xq); free(xb);
    if (converged) *converged = ok;
    return it;
}

/* ---------------------------------------------------------------------------
 * The time-stepping state.
 * ------------------------------------------------------------------------- */
enum { BC_ZOU_HE = 0, BC_PERIODIC = 1 };
enum { ERR_UNSTABLE = 1, ERR_NOCONV = 2, ERR_WALL = 4 };

typedef struct {
    int n[3], bc[3], rule;
    double tau;
    size_t nn;
    double *f, *fn;      /* [Q][nn] pre-collision populations f_t(x) */
    double *F;           /* [3][nn] Eulerian force of the last step */
    double *rho, *u;     /* [nn], [3][nn] moments of the last step */
    double *frames;      /* [n_frames][3][3], A[a][b] = du_a/dx_b */
    int n_frames, n_hold;
    long step;
    int err;
    /* mesh (optional) */
    int nv, nt;
    double *r, *Fn;
    int *tri;
    double sigma;
    int *nb_ptr, *nb_idx;
    int reg_every, reg_max_iter, reg_plus, reg_last_iters, reg_keep_volume;
    double reg_alpha, reg_gamma, reg_tol;
    /* re-centring: the linear boundary field is centred on the droplet's
     * centre of mass at the start of each step instead of the box centre */
    int recentre;
    double centre[3];
    /* viscosity ratio: tau_in inside the droplet (chi != 1 only) */
    int visc;
    double tau_in;
    unsigned char *ind; /* [nn] 1 inside the droplet at the current step */
} orc_sim;

static size_t nid(const orc_sim *s, int x, int y, int z)
{
    return (size_t)x + (size_t)s->n[0] * ((size_t)y + (size_t)s->n[1] * (size_t)z);
}

static const double *frame_of(const orc_sim *s, long t)
{
    long k = t / s->n_hold;
    if (k > s->n_frames - 1) k = s->n_frames - 1;
    return s->frames + 9 * k;
}

/* Eq. (velo_facce_cubo_da_gradiente): u_a = sum_b A_ab (l_b - L_b/2), with
 * L_b = n_b - 1 the side length between the two wet boundary planes.  With
 * re-centring, L_b/2 is replaced by the droplet's centre of mass (the
 * Sec. 3.2 remark that the linearisation is centred there). */
static void wall_velocity(const orc_sim *s, const double *A, int x, int y, int z, double uw[3])
{
    double l[3];
    if (s->recentre) {
        l[0] = x - s->centre[0];
        l[1] = y - s->centre[1];
        l[2] = z - s->centre[2];
    } else {
        l[0] = x - 0.5 * (s->n[0] - 1);
        l[1] = y - 0.5 * (s->n[1] - 1);
        l[2] = z - 0.5 * (s->n[2] - 1);
    }
    for (int a = 0; a < 3; ++a) uw[a] = A[3 * a] * l[0] + A[3 * a + 1] * l[1] + A[3 * a + 2] * l[2];
}

orc_sim *orc_sim_create(const int n[3], const int bc[3], double tau, int rule,
                        const double *frames, int n_frames, int n_hold)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    for (int a = 0; a < 3; ++a) { s->n[a] = n[a]; s->bc[a] = bc[a]; }
    s->tau = tau;
    s->rule = rule;
    s->nn = (size_t)n[0] * n[1] * n[2];
    s->f = (double *)calloc(Q * s->nn, sizeof(double));
    s->fn = (double *)calloc(Q * s->nn, sizeof(double));
    s->F = (double *)calloc(3 * s->nn, sizeof(double));
    s->rho = (double *)calloc(s->nn, sizeof(double));
    s->u = (double *)calloc(3 * s->nn, sizeof(double));
    s->n_frames = n_frames;
    s->n_hold = n_hold > 0 ? n_hold : 1;
    s->frames = (double *)malloc(sizeof(double) * 9 * (size_t)n_frames);
    memcpy(s->frames, frames, sizeof(double) * 9 * (size_t)n_frames);
    s->reg_alpha = 0.1; s->reg_gamma = 0.51; s->reg_tol = 0.01; s->reg_max_iter = 100;
    s->reg_plus = 1;
    /* initial state: f = f_eq(rho = 1, u = A(0)(x - c)) at every node */
    const double *A0 = frame_of(s, 0);
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x) {
                double u0[3], feq[Q];
                wall_velocity(s, A0, x, y, z, u0);
                orc_equilibrium(1.0, u0, feq);
                size_t id = nid(s, x, y, z);
                for (int i = 0; i < Q; ++i) s->f[i * s->nn + id] = feq[i];
            }
    return s;
}

void orc_sim_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->f); free(s->fn); free(s->F); free(s->rho); free(s->u); free(s->frames);
    free(s->r); free(s->Fn); free(s->tri); free(s->nb_ptr); free(s->nb_idx);
    free(s->ind);
    free(s);
}

int orc_sim_set_mesh(orc_sim *s, int nv, const double *r, int nt, const int *tri, double sigma,
                     const int *nb_ptr, const int *nb_idx)
{
    free(s->r); free(s->Fn); free(s->tri); free(s->nb_ptr); free(s->nb_idx);
    s->nv = nv; s->nt = nt; s->sigma = sigma;
    s->r = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    s->Fn = (double *)calloc(3 * (size_t)nv, sizeof(double));
    s->tri = (int *)malloc(sizeof(int) * 3 * (size_t)nt);
    memcpy(s->r, r, sizeof(double) * 3 * (size_t)nv);
    memcpy(s->tri, tri, sizeof(int) * 3 * (size_t)nt);
    s->nb_ptr = (int *)malloc(sizeof(int) * (size_t)(nv + 1));
    memcpy(s->nb_ptr, nb_ptr, sizeof(int) * (size_t)(nv + 1));
    s->nb_idx = (int *)malloc(sizeof(int) * (size_t)nb_ptr[nv]);
    memcpy(s->nb_idx, nb_idx, sizeof(int) * (size_t)nb_ptr[nv]);
    return 0;
}

void orc_sim_set_regularization(orc_sim *s, double alpha, double gamma, double tol, int max_iter,
                                int every, int plus_sign)
{
    s->reg_alpha = alpha; s->reg_gamma = gamma; s->reg_tol = tol;
    s->reg_max_iter = max_iter; s->reg_every = every; s->reg_plus = plus_sign;
}

/* keep = 1: every regularisation is followed by orc_restore_volume to the
 * volume enclosed before it (an option beyond Sec. 3.3). */
void orc_sim_set_regularization_volume(orc_sim *s, int keep) { s->reg_keep_volume = keep; }

/* Re-centring on (1) or off (0); needs a droplet mesh to take effect. */
void orc_sim_set_recentring(orc_sim *s, int on) { s->recentre = on; }

/* ---------------------------------------------------------------------------
 * Viscosity ratio (Sec. 2: the droplet phase has viscosity chi mu, the carrier
 * mu).  With equal densities the relaxation time inside the droplet is
 * tau_in = 1/2 + chi (tau - 1/2).  Inside is decided per lattice node by the
 * even-odd rule on a vertical ray: node (x, y, z) is inside when the number
 * of triangles crossed strictly above it is odd.  Triangle (a, b, c) is
 * crossed above the node when q = (x + RAY_DX, y + RAY_DY) lies strictly
 * inside its projection on the xy plane (all three edge functions of one
 * sign) and its height over q, interpolated with the barycentric weights,
 * exceeds z.  The fixed sub-lattice offsets keep the rays off the mesh's
 * vertices and edges.  Every product and sum is a separate IEEE operation
 * (this file is compiled without contraction), in the order written.
 */
static const double RAY_DX = 1.4142135623730951e-7, RAY_DY = 1.7320508075688772e-7;

void orc_indicator(const int n[3], int nv, const double *r, int nt, const int *tri, unsigned char *ind)
{
    (void)nv;
    const size_t nn = (size_t)n[0] * n[1] * n[2];
    memset(ind, 0, nn);
    for (int t = 0; t < nt; ++t) {
        const double *a = r + 3 * tri[3 * t], *b = r + 3 * tri[3 * t + 1], *c = r + 3 * tri[3 * t + 2];
        const double xmin = fmin(a[0], fmin(b[0], c[0])), xmax = fmax(a[0], fmax(b[0], c[0]));
        const double ymin = fmin(a[1], fmin(b[1], c[1])), ymax = fmax(a[1], fmax(b[1], c[1]));
        int x0 = (int)ceil(xmin - RAY_DX), x1 = (int)floor(xmax - RAY_DX);
        int y0 = (int)ceil(ymin - RAY_DY), y1 = (int)floor(ymax - RAY_DY);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > n[0] - 1) x1 = n[0] - 1;
        if (y1 > n[1] - 1) y1 = n[1] - 1;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                const double qx = (double)x + RAY_DX, qy = (double)y + RAY_DY;
                const double e0 = (b[0] - a[0]) * (qy - a[1]) - (b[1] - a[1]) * (qx - a[0]);
                const double e1 = (c[0] - b[0]) * (qy - b[1]) - (c[1] - b[1]) * (qx - b[0]);
                const double e2 = (a[0] - c[0]) * (qy - c[1]) - (a[1] - c[1]) * (qx - c[0]);
                const int inside = (e0 > 0.0 && e1 > 0.0 && e2 > 0.0) || (e0 < 0.0 && e1 < 0.0 && e2 < 0.0);
                if (!inside) continue;
                const double zc = ((e1 * a[2] + e2 * b[2]) + e0 * c[2]) / ((e0 + e1) + e2);
                for (int z = 0; z < n[2]; ++z)
                    if ((double)z < zc) ind[(size_t)x + (size_t)n[0] * ((size_t)y + (size_t)n[1] * z)] ^= 1;
            }
    }
}

/* chi = 1 switches the viscosity ratio off.  Needs a mesh and Zou-He walls on
 * every axis (a vertical ray must not wrap); returns 0 otherwise. */
int orc_sim_set_viscosity_ratio(orc_sim *s, double chi)
{
    if (!(chi > 0.0) || s->nv <= 0) return 0;
    for (int a = 0; a < 3; ++a)
        if (s->bc[a] != BC_ZOU_HE) return 0;
    s->visc = chi != 1.0;
    s->tau_in = 0.5 + chi * (s->tau - 0.5);
    if (!s->ind) s->ind = (unsigned char *)calloc(s->nn, 1);
    return 1;
}

void orc_sim_get_indicator(const orc_sim *s, unsigned char *out)
{
    if (s->ind) memcpy(out, s->ind, s->nn);
    else memset(out, 0, s->nn);
}

/* Centre of the linear boundary field used by the last step. */
void orc_sim_get_centre(const orc_sim *s, double c[3])
{
    for (int a = 0; a < 3; ++a) c[a] = s->centre[a];
}

/* Stencil of the 4-point kernel along axis a around coordinate ra: the four
 * nodes floor(ra)-1 .. floor(ra)+2 with their weights.  On a Zou-He axis all
 * four must be interior nodes (1 .. n-2), so that no force reaches the wet
 * boundary nodes; periodic axes wrap.  Returns 0 if the stencil is invalid. */
static int stencil(const orc_sim *s, int a, double ra, int idx[4], double w[4])
{
    if (!(ra == ra)) return 0; /* NaN */
    double fl = floor(ra);
    if (fl < -1e9 || fl > 1e9) return 0;
    int base = (int)fl - 1;
    for (int k = 0; k < 4; ++k) {
        int g = base + k;
        w[k] = orc_peskin_phi(ra - (double)g);
        if (s->bc[a] == BC_PERIODIC) {
            g %= s->n[a];
            if (g < 0) g += s->n[a];
        } else if (g < 1 || g > s->n[a] - 2) {
            return 0;
        }
        idx[k] = g;
    }
    return 1;
}

/* Eq. (ibm_force_d)(a): F_ext(x) = sum_i phi_i Delta(r_i - x), serial in node order. */
static void spread(orc_sim *s)
{
    memset(s->F, 0, sizeof(double) * 3 * s->nn);
    orc_nodal_forces(s->nv, s->r, s->nt, s->tri, s->sigma, s->Fn);
    for (int i = 0; i < s->nv; ++i) {
        int ix[4], iy[4], iz[4];
        double wx[4], wy[4], wz[4];
        if (!stencil(s, 0, s->r[3 * i], ix, wx) || !stencil(s, 1, s->r[3 * i + 1], iy, wy) ||
            !stencil(s, 2, s->r[3 * i + 2], iz, wz)) {
            s->err |= ERR_WALL;
            continue;
        }
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    double d = wx[a] * wy[b] * wz[c];
                    size_t id = nid(s, ix[a], iy[b], iz[c]);
                    for (int k = 0; k < 3; ++k) s->F[k * s->nn + id] += s->Fn[3 * i + k] * d;
                }
    }
}

/* Eq. (ibm_force_d)(b) and Eq. (fwd_euler): r_i <- r_i + sum_x u(x) Delta(r_i - x). */
static void interpolate_advect(orc_sim *s)
{
    for (int i = 0; i < s->nv; ++i) {
        int ix[4], iy[4], iz[4];
        double wx[4], wy[4], wz[4];
        if (!stencil(s, 0, s->r[3 * i], ix, wx) || !stencil(s, 1, s->r[3 * i + 1], iy, wy) ||
            !stencil(s, 2, s->r[3 * i + 2], iz, wz)) {
            s->err |= ERR_WALL;
            continue;
        }
        double v[3] = {0, 0, 0};
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    double d = wx[a] * wy[b] * wz[c];
                    size_t id = nid(s, ix[a], iy[b], iz[c]);
                    for (int k = 0; k < 3; ++k) v[k] += s->u[k * s->nn + id] * d;
                }
        for (int k = 0; k < 3; ++k) s->r[3 * i + k] += v[k];
    }
}

/* One lattice update: boundary reconstruction, moments, BGK + Guo, push streaming. */
static void lattice_update(orc_sim *s)
{
    const double *A = frame_of(s, s->step);
    const double tau = s->tau;
    const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
    int unstable = 0;
#pragma omp parallel for schedule(static) reduction(| : unstable)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t id = nid(s, x, y, z);
                double f[Q];
                for (int i = 0; i < Q; ++i) f[i] = s->f[i * s->nn + id];
                int side[3] = {0, 0, 0};
                const int c[3] = {x, y, z};
                for (int a = 0; a < 3; ++a)
                    if (s->bc[a] == BC_ZOU_HE) side[a] = (c[a] == 0) ? -1 : (c[a] == s->n[a] - 1 ? 1 : 0);
                if (side[0] || side[1] || side[2]) {
                    double uw[3];
                    wall_velocity(s, A, x, y, z, uw);
                    orc_bc_node(f, side, uw, s->rule);
                }
                const double tau_x = (s->visc && s->ind[id]) ? s->tau_in : tau;
                double Fx[3] = {s->F[id], s->F[s->nn + id], s->F[2 * s->nn + id]};
                double rho = 0.0, j[3] = {0, 0, 0};
                for (int i = 0; i < Q; ++i) {
                    rho += f[i];
                    for (int a = 0; a < 3; ++a) j[a] += CV[i][a] * f[i];
                }
                double u[3];
                for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * Fx[a]) / rho;
                if (!(rho == rho) || u[0] * u[0] + u[1] * u[1] + u[2] * u[2] > 0.09) unstable = 1;
                s->rho[id] = rho;
                for (int a = 0; a < 3; ++a) s->u[a * s->nn + id] = u[a];
                double feq[Q], S[Q];
                orc_equilibrium(rho, u, feq);
                orc_guo_source(tau_x, u, Fx, S);
                for (int i = 0; i < Q; ++i) {
                    double fs = f[i] - (f[i] - feq[i]) / tau_x + S[i];
                    int d[3];
                    int inside = 1;
                    for (int a = 0; a < 3; ++a) {
                        d[a] = c[a] + CV[i][a];
                        if (s->bc[a] == BC_PERIODIC) {
                            d[a] = (d[a] + s->n[a]) % s->n[a];
                        } else if (d[a] < 0 || d[a] >= s->n[a]) {
                            inside = 0;
                        }
                    }
                    if (inside) s->fn[i * s->nn + nid(s, d[0], d[1], d[2])] = fs;
                }
            }
    }
    if (unstable) s->err |= ERR_UNSTABLE;
    double *t = s->f;
    s->f = s->fn;
    s->fn = t;
}

/* Centre of the boundary field for the step about to run: the droplet's
 * centre of mass (the volume centroid of the closed mesh) at r_t with
 * re-centring, else the box centre. */
static void step_centre(orc_sim *s)
{
    if (s->recentre && s->nv > 0) {
        double V;
        orc_enclosed_volume(s->nv, s->r, s->nt, s->tri, &V, s->centre);
    } else {
        for (int a = 0; a < 3; ++a) s->centre[a] = 0.5 * (s->n[a] - 1);
    }
}

/* One IBLB step in the order: forces + spread at r_t, lattice update with
 * F_t, interpolation of u_t at r_t and advection, regularisation when
 * scheduled.  Returns the sticky error bits. */
int orc_sim_step(orc_sim *s, long nsteps)
{
    for (long k = 0; k < nsteps; ++k) {
        step_centre(s);
        if (s->visc) orc_indicator(s->n, s->nv, s->r, s->nt, s->tri, s->ind);
        if (s->nv > 0) spread(s);
        else memset(s->F, 0, sizeof(double) * 3 * s->nn);
        lattice_update(s);
        if (s->nv > 0) {
            interpolate_advect(s);
            if (s->reg_every > 0 && (s->step + 1) % s->reg_every == 0) {
                int conv = 0;
                double V0 = 0.0, c0[3];
                if (s->reg_keep_volume) orc_enclosed_volume(s->nv, s->r, s->nt, s->tri, &V0, c0);
                s->reg_last_iters = orc_regularize(s->nv, s->r, s->nb_ptr, s->nb_idx, s->reg_alpha,
                                                   s->reg_gamma, s->reg_tol, s->reg_max_iter,
                                                   s->reg_plus, &conv);
                if (s->reg_keep_volume) orc_restore_volume(s->nv, s->r, s->nt, s->tri, V0);
                if (!conv) s->err |= ERR_NOCONV;
            }
        }
        s->step += 1;
    }
    return s->err;
}

/* Same step with a uniform body force g added to the Eulerian force of every
 * node that is not a wet boundary node (used by the Poiseuille pin). */
int orc_sim_step_body_force(orc_sim *s, long nsteps, const double g[3])
{
    for (long k = 0; k < nsteps; ++k) {
        step_centre(s);
        if (s->nv > 0) spread(s);
        else memset(s->F, 0, sizeof(double) * 3 * s->nn);
        for (int z = 0; z < s->n[2]; ++z)
            for (int y = 0; y < s->n[1]; ++y)
                for (int x = 0; x < s->n[0]; ++x) {
                    const int c[3] = {x, y, z};
                    int wet = 0;
                    for (int a = 0; a < 3; ++a)
                        if (s->bc[a] == BC_ZOU_HE && (c[a] == 0 || c[a] == s->n[a] - 1)) wet = 1;
                    if (wet) continue;
                    size_t id = nid(s, x, y, z);
                    for (int a = 0; a < 3; ++a) s->F[a * s->nn + id] += g[a];
                }
        lattice_update(s);
        if (s->nv > 0) interpolate_advect(s);
        s->step += 1;
    }
    return s->err;
}

long orc_sim_get_step(const orc_sim *s) { return s->step; }
int orc_sim_get_error(const orc_sim *s) { return s->err; }
int orc_sim_get_reg_iters(const orc_sim *s) { return s->reg_last_iters; }

void orc_sim_get_fields(const orc_sim *s, double *rho, double *u, double *F)
{
    if (rho) memcpy(rho, s->rho, sizeof(double) * s->nn);
    if (u) memcpy(u, s->u, sizeof(double) * 3 * s->nn);
    if (F) memcpy(F, s->F, sizeof(double) * 3 * s->nn);
}

void orc_sim_get_mesh(const orc_sim *s, double *r, double *Fn)
{
    if (r) memcpy(r, s->r, sizeof(double) * 3 * (size_t)s->nv);
    if (Fn) memcpy(Fn, s->Fn, sizeof(double) * 3 * (size_t)s->nv);
}

void orc_sim_set_positions(orc_sim *s, const double *r)
{
    memcpy(s->r, r, sizeof(double) * 3 * (size_t)s->nv);
}

/* Current pre-collision state f_t(x), with the populations that a boundary
 * node has no source for (unknown until reconstructed) set to zero. */
void orc_sim_get_populations(const orc_sim *s, double *out)
{
    for (int z = 0; z < s->n[2]; ++z)
        for (int y = 0; y < s->n[1]; ++y)
            for (int x = 0; x < s->n[0]; ++x) {
                size_t id = nid(s, x, y, z);
                int side[3] = {0, 0, 0};
                const int c[3] = {x, y, z};
                for (int a = 0; a < 3; ++a)
                    if (s->bc[a] == BC_ZOU_HE) side[a] = (c[a] == 0) ? -1 : (c[a] == s->n[a] - 1 ? 1 : 0);
                for (int i = 0; i < Q; ++i)
                    out[i * s->nn + id] = unknown(i, side) ? 0.0 : s->f[i * s->nn + id];
            }
}

void orc_sim_set_populations(orc_sim *s, const double *in, long step)
{
    memcpy(s->f, in, sizeof(double) * Q * s->nn);
    s->step = step;
}
