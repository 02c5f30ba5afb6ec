/*
 * Oracle: plain, slow, obviously-correct FP64 reference for the stencil/RK4
 * level path.  TEST INFRASTRUCTURE ONLY: it is called from tests/, from the
 * package's smoke check and from bench.py's CPU-baseline leg, never from the
 * product path.  It shares no code, header or constant generator with the
 * CUDA library.
 *
 * Compiled with -O2 -ffp-contract=off so that every a*b+c is two roundings,
 * in the order written here.  The optional OpenMP pragmas only split the
 * outermost z loop; each point's arithmetic is unchanged, so results are
 * bit-identical for any thread count.
 *
 * What it computes (the equations are restated here, not copied):
 *
 *  - The level is a set of boxes on a uniform grid whose points are
 *    x0 + n*h with integer n (paper Sec. 2, "Efficient Bounding Box
 *    Algebra").  Each box carries ghost zones of width 2; a ghost point takes
 *    the value of the unique interior point of the level that it coincides
 *    with (periodic images included).  This is the communication schedule the
 *    paper derives from bboxsets (Sec. 2, list of operations built on the
 *    set algebra).
 *
 *  - The spatial operator is the 4th-order centred second difference, summed
 *    over the three axes, applied to padded arrays in the manner of the
 *    paper's centred-difference example (Sec. 4.3, "Iterators"):
 *        (L u)_i = sum_d ( -u_{i-2e_d} + 16 u_{i-e_d} - 30 u_i
 *                          + 16 u_{i+e_d} - u_{i+2e_d} ) / (12 h^2)
 *
 *  - The PDE is the first-order-in-time scalar wave equation
 *        du/dt = pi,   dpi/dt = c2(x) * (L u),
 *    i.e. y' = A y with A(u, pi) = (pi, c2 * L u), integrated by the classic
 *    fourth-order Runge-Kutta method (nodes 0, 1/2, 1/2, 1; weights
 *    1/6, 1/3, 1/3, 1/6) in its plain stage form.
 *
 *  - The tangent-linear and adjoint of one RK4 step (with respect to the
 *    state and to c2), and the checkpointed reverse sweep that gives the
 *    gradient of a loss of the final state.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

static int g_threads = 1;

/* Number of OpenMP threads used by the loops below (1 = serial). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n < 1) n = 1;
    g_threads = n;
    omp_set_num_threads(n);
    return n;
#else
    (void)n;
    g_threads = 1;
    return 1;
#endif
}

int oracle_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* Periodic index wrap: the unique j in [0, n) with j == i (mod n). */
static i64 wrap(i64 i, i64 n)
{
    i64 j = i % n;
    return j < 0 ? j + n : j;
}

/* ------------------------------------------------------------------------ */
/* Laplacian                                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Periodic 4th-order Laplacian on a whole periodic domain.
 * u, out: arrays of nx*ny*nz doubles, index (k*ny + j)*nx + i (x fastest).
 */
void oracle_lap_periodic(const double *u, double *out,
                         i64 nx, i64 ny, i64 nz, double h)
{
    const double inv = 1.0 / (12.0 * h * h);
    i64 k;
#pragma omp parallel for schedule(static) if (g_threads > 1)
    for (k = 0; k < nz; ++k) {
        for (i64 j = 0; j < ny; ++j) {
            for (i64 i = 0; i < nx; ++i) {
#define U(ii, jj, kk) u[(wrap(kk, nz) * ny + wrap(jj, ny)) * nx + wrap(ii, nx)]
                double c = U(i, j, k);
                double dxx = -U(i - 2, j, k) + 16.0 * U(i - 1, j, k) - 30.0 * c
                             + 16.0 * U(i + 1, j, k) - U(i + 2, j, k);
                double dyy = -U(i, j - 2, k) + 16.0 * U(i, j - 1, k) - 30.0 * c
                             + 16.0 * U(i, j + 1, k) - U(i, j + 2, k);
                double dzz = -U(i, j, k - 2) + 16.0 * U(i, j, k - 1) - 30.0 * c
                             + 16.0 * U(i, j, k + 1) - U(i, j, k + 2);
#undef U
                out[(k * ny + j) * nx + i] = (dxx + dyy + dzz) * inv;
            }
        }
    }
}

/*
 * Same operator on one padded box: up has (nz+4)*(ny+4)*(nx+4) doubles with
 * ghost width 2 on every side (dense, x fastest); out receives the nx*ny*nz
 * interior values.  Ghosts are whatever the caller put there (used by the
 * polynomial-exactness checks, which fill them by evaluating the polynomial).
 */
void oracle_lap_padded(const double *up, double *out,
                       i64 nx, i64 ny, i64 nz, double h)
{
    const double inv = 1.0 / (12.0 * h * h);
    const i64 px = nx + 4, py = ny + 4;
    i64 k;
#pragma omp parallel for schedule(static) if (g_threads > 1)
    for (k = 0; k < nz; ++k) {
        for (i64 j = 0; j < ny; ++j) {
            for (i64 i = 0; i < nx; ++i) {
#define P(ii, jj, kk) up[((kk + 2) * py + (jj + 2)) * px + (ii + 2)]
                double c = P(i, j, k);
                double dxx = -P(i - 2, j, k) + 16.0 * P(i - 1, j, k) - 30.0 * c
                             + 16.0 * P(i + 1, j, k) - P(i + 2, j, k);
                double dyy = -P(i, j - 2, k) + 16.0 * P(i, j - 1, k) - 30.0 * c
                             + 16.0 * P(i, j + 1, k) - P(i, j + 2, k);
                double dzz = -P(i, j, k - 2) + 16.0 * P(i, j, k - 1) - 30.0 * c
                             + 16.0 * P(i, j, k + 1) - P(i, j, k + 2);
#undef P
                out[(k * ny + j) * nx + i] = (dxx + dyy + dzz) * inv;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Classic RK4 on a whole periodic domain                                     */
/* ------------------------------------------------------------------------ */

/* Runge-Kutta nodes a_s (stage s input is y + a_s*dt*K_{s-1}) and weights. */
static const double RK_A[4] = {0.0, 0.5, 0.5, 1.0};
static const double RK_B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

static double *alloc_d(i64 n)
{
    double *p = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    return p;
}

/*
 * nsteps classic RK4 steps of y' = A y, A(u, pi) = (pi, c2 * L u), in place
 * on u and pi (each nx*ny*nz, periodic).  Stage form:
 *   Y_1 = y,  K_s = A Y_s,  Y_{s+1} = y + a_{s+1} dt K_s,
 *   y_new = y + dt (K_1 + 2 K_2 + 2 K_3 + K_4) / 6.
 * Returns 0, or -1 if a temporary could not be allocated.
 */
int oracle_rk4_periodic(double *u, double *pi, const double *c2,
                        i64 nx, i64 ny, i64 nz, double h, double dt,
                        i64 nsteps)
{
    const i64 n = nx * ny * nz;
    double *Ku[4], *Kp[4];
    double *Yu = alloc_d(n), *Yp = alloc_d(n), *lap = alloc_d(n);
    int ok = Yu && Yp && lap;
    for (int s = 0; s < 4; ++s) {
        Ku[s] = alloc_d(n);
        Kp[s] = alloc_d(n);
        ok = ok && Ku[s] && Kp[s];
    }
    if (!ok) {
        free(Yu); free(Yp); free(lap);
        for (int s = 0; s < 4; ++s) { free(Ku[s]); free(Kp[s]); }
        return -1;
    }
    for (i64 step = 0; step < nsteps; ++step) {
        memcpy(Yu, u, (size_t)n * sizeof(double));
        memcpy(Yp, pi, (size_t)n * sizeof(double));
        for (int s = 0; s < 4; ++s) {
            oracle_lap_periodic(Yu, lap, nx, ny, nz, h);
            i64 i;
#pragma omp parallel for schedule(static) if (g_threads > 1)
            for (i = 0; i < n; ++i) {
                Ku[s][i] = Yp[i];
                Kp[s][i] = c2[i] * lap[i];
            }
            if (s < 3) {
                const double a = RK_A[s + 1] * dt;
#pragma omp parallel for schedule(static) if (g_threads > 1)
                for (i = 0; i < n; ++i) {
                    Yu[i] = u[i] + a * Ku[s][i];
                    Yp[i] = pi[i] + a * Kp[s][i];
                }
            }
        }
        i64 i;
#pragma omp parallel for schedule(static) if (g_threads > 1)
        for (i = 0; i < n; ++i) {
            u[i] = u[i] + dt * (Ku[0][i] + 2.0 * Ku[1][i] + 2.0 * Ku[2][i] + Ku[3][i]) / 6.0;
            pi[i] = pi[i] + dt * (Kp[0][i] + 2.0 * Kp[1][i] + 2.0 * Kp[2][i] + Kp[3][i]) / 6.0;
        }
    }
    free(Yu); free(Yp); free(lap);
    for (int s = 0; s < 4; ++s) { free(Ku[s]); free(Kp[s]); }
    return 0;
}

/*
 * One classic RK4 step on ONE padded box whose ghost ring holds boundary
 * values (ghost width 2 on every side; u, pi, c2 dense, (nz+4)(ny+4)(nx+4),
 * x fastest).  The ghost values of every stage input Y_s.u are those of u at
 * the start of the step (boundary data held fixed over the step); only the
 * interior of u and pi changes.  The stage expressions and their order are
 * those of oracle_rk4_periodic, so interior points whose dependence cone
 * stays inside the box get the same bits as a periodic run.
 * Returns 0, or -1 if a temporary could not be allocated.
 */
int oracle_rk4_padded(double *u, double *pi, const double *c2,
                      i64 nx, i64 ny, i64 nz, double h, double dt)
{
    const i64 px = nx + 4, py = ny + 4, pz = nz + 4;
    const i64 n = nx * ny * nz, np = px * py * pz;
    double *Ku[4], *Kp[4];
    double *Yu = alloc_d(np), *Yp = alloc_d(n), *lap = alloc_d(n);
    int ok = Yu && Yp && lap;
    for (int s = 0; s < 4; ++s) {
        Ku[s] = alloc_d(n);
        Kp[s] = alloc_d(n);
        ok = ok && Ku[s] && Kp[s];
    }
    if (!ok) {
        free(Yu); free(Yp); free(lap);
        for (int s = 0; s < 4; ++s) { free(Ku[s]); free(Kp[s]); }
        return -1;
    }
#define IP(ii, jj, kk) ((((kk) + 2) * py + ((jj) + 2)) * px + ((ii) + 2))
    memcpy(Yu, u, (size_t)np * sizeof(double));
    for (i64 k = 0; k < nz; ++k)
        for (i64 j = 0; j < ny; ++j)
            for (i64 i = 0; i < nx; ++i)
                Yp[(k * ny + j) * nx + i] = pi[IP(i, j, k)];
    for (int s = 0; s < 4; ++s) {
        oracle_lap_padded(Yu, lap, nx, ny, nz, h);
        for (i64 k = 0; k < nz; ++k)
            for (i64 j = 0; j < ny; ++j)
                for (i64 i = 0; i < nx; ++i) {
                    const i64 q = (k * ny + j) * nx + i;
                    Ku[s][q] = Yp[q];
                    Kp[s][q] = c2[IP(i, j, k)] * lap[q];
                }
        if (s < 3) {
            const double a = RK_A[s + 1] * dt;
            for (i64 k = 0; k < nz; ++k)
                for (i64 j = 0; j < ny; ++j)
                    for (i64 i = 0; i < nx; ++i) {
                        const i64 q = (k * ny + j) * nx + i, g = IP(i, j, k);
                        Yu[g] = u[g] + a * Ku[s][q];
                        Yp[q] = pi[g] + a * Kp[s][q];
                    }
        }
    }
    for (i64 k = 0; k < nz; ++k)
        for (i64 j = 0; j < ny; ++j)
            for (i64 i = 0; i < nx; ++i) {
                const i64 q = (k * ny + j) * nx + i, g = IP(i, j, k);
                u[g] = u[g] + dt * (Ku[0][q] + 2.0 * Ku[1][q] + 2.0 * Ku[2][q] + Ku[3][q]) / 6.0;
                pi[g] = pi[g] + dt * (Kp[0][q] + 2.0 * Kp[1][q] + 2.0 * Kp[2][q] + Kp[3][q]) / 6.0;
            }
#undef IP
    free(Yu); free(Yp); free(lap);
    for (int s = 0; s < 4; ++s) { free(Ku[s]); free(Kp[s]); }
    return 0;
}

/*
 * Discrete energy E = 1/2 sum( pi^2 / c2 - u * (L u) ) h^3 over the periodic
 * domain.  For c2 > 0 and the symmetric negative semi-definite L this is a
 * non-negative quadratic form, conserved by the semi-discrete system.
 */
double oracle_energy_periodic(const double *u, const double *pi, const double *c2,
                              i64 nx, i64 ny, i64 nz, double h)
{
    const i64 n = nx * ny * nz;
    double *lap = alloc_d(n);
    if (!lap) return NAN;
    oracle_lap_periodic(u, lap, nx, ny, nz, h);
    double e = 0.0;
    for (i64 i = 0; i < n; ++i)
        e += pi[i] * pi[i] / c2[i] - u[i] * lap[i];
    free(lap);
    return 0.5 * e * h * h * h;
}

/* ------------------------------------------------------------------------ */
/* Tangent-linear RK4 step (forward mode), used only to check the adjoint     */
/* ------------------------------------------------------------------------ */

/*
 * Advances (u, pi) by nsteps RK4 steps and, alongside, the tangent
 * (du, dpi) of the state in the direction (du, dpi, dc2):
 *   dK_s = ( dY_s^pi , c2 * L dY_s^u + dc2 * L Y_s^u ),
 *   dY_{s+1} = dy + a_{s+1} dt dK_s,   dy_new = dy + dt sum_s b_s dK_s.
 * All arrays nx*ny*nz, periodic; updated in place.
 */
int oracle_tlm_periodic(double *u, double *pi, const double *c2,
                        double *du, double *dpi, const double *dc2,
                        i64 nx, i64 ny, i64 nz, double h, double dt,
                        i64 nsteps)
{
    const i64 n = nx * ny * nz;
    double *Ku[4], *Kp[4], *dKu[4], *dKp[4];
    double *Yu = alloc_d(n), *Yp = alloc_d(n), *dYu = alloc_d(n), *dYp = alloc_d(n);
    double *lap = alloc_d(n), *dlap = alloc_d(n);
    int ok = Yu && Yp && dYu && dYp && lap && dlap;
    for (int s = 0; s < 4; ++s) {
        Ku[s] = alloc_d(n); Kp[s] = alloc_d(n);
        dKu[s] = alloc_d(n); dKp[s] = alloc_d(n);
        ok = ok && Ku[s] && Kp[s] && dKu[s] && dKp[s];
    }
    if (ok) {
        for (i64 step = 0; step < nsteps; ++step) {
            memcpy(Yu, u, (size_t)n * sizeof(double));
            memcpy(Yp, pi, (size_t)n * sizeof(double));
            memcpy(dYu, du, (size_t)n * sizeof(double));
            memcpy(dYp, dpi, (size_t)n * sizeof(double));
            for (int s = 0; s < 4; ++s) {
                oracle_lap_periodic(Yu, lap, nx, ny, nz, h);
                oracle_lap_periodic(dYu, dlap, nx, ny, nz, h);
                for (i64 i = 0; i < n; ++i) {
                    Ku[s][i] = Yp[i];
                    Kp[s][i] = c2[i] * lap[i];
                    dKu[s][i] = dYp[i];
                    dKp[s][i] = c2[i] * dlap[i] + dc2[i] * lap[i];
                }
                if (s < 3) {
                    const double a = RK_A[s + 1] * dt;
                    for (i64 i = 0; i < n; ++i) {
                        Yu[i] = u[i] + a * Ku[s][i];
                        Yp[i] = pi[i] + a * Kp[s][i];
                        dYu[i] = du[i] + a * dKu[s][i];
                        dYp[i] = dpi[i] + a * dKp[s][i];
                    }
                }
            }
            for (i64 i = 0; i < n; ++i) {
                u[i] = u[i] + dt * (Ku[0][i] + 2.0 * Ku[1][i] + 2.0 * Ku[2][i] + Ku[3][i]) / 6.0;
                pi[i] = pi[i] + dt * (Kp[0][i] + 2.0 * Kp[1][i] + 2.0 * Kp[2][i] + Kp[3][i]) / 6.0;
                du[i] = du[i] + dt * (dKu[0][i] + 2.0 * dKu[1][i] + 2.0 * dKu[2][i] + dKu[3][i]) / 6.0;
                dpi[i] = dpi[i] + dt * (dKp[0][i] + 2.0 * dKp[1][i] + 2.0 * dKp[2][i] + dKp[3][i]) / 6.0;
            }
        }
    }
    free(Yu); free(Yp); free(dYu); free(dYp); free(lap); free(dlap);
    for (int s = 0; s < 4; ++s) { free(Ku[s]); free(Kp[s]); free(dKu[s]); free(dKp[s]); }
    return ok ? 0 : -1;
}

/* ------------------------------------------------------------------------ */
/* Adjoint (reverse mode) of one RK4 step                                      */
/* ------------------------------------------------------------------------ */

/*
 * One reverse step.  (u, pi) is the state at the START of the step (it is
 * not modified); (bu, bpi) holds on entry the adjoint of the step's output
 * and on return the adjoint of its input; bc2 accumulates the c2 adjoint.
 *
 * The forward stages are recomputed to get L U_s.  With
 * A^T(ab, bb) = ( L(c2 * bb), ab )  (L is symmetric on a periodic grid):
 *   Kb_s = b_s dt yb_out  for all s,  yb = yb_out;
 *   for s = 4..1:
 *     Yb_s  = A^T Kb_s;   c2b += Kb_s^pi * L U_s;   yb += Yb_s;
 *     if s > 1: Kb_{s-1} += a_s dt Yb_s.
 */
int oracle_adj_step_periodic(const double *u, const double *pi, const double *c2,
                             double *bu, double *bpi, double *bc2,
                             i64 nx, i64 ny, i64 nz, double h, double dt)
{
    const i64 n = nx * ny * nz;
    double *lapU[4], *Kbu[4], *Kbp[4];
    double *Yu = alloc_d(n), *Yp = alloc_d(n), *Ku = alloc_d(n), *Kp = alloc_d(n);
    double *t = alloc_d(n), *lt = alloc_d(n), *ybu = alloc_d(n), *ybp = alloc_d(n);
    int ok = Yu && Yp && Ku && Kp && t && lt && ybu && ybp;
    for (int s = 0; s < 4; ++s) {
        lapU[s] = alloc_d(n); Kbu[s] = alloc_d(n); Kbp[s] = alloc_d(n);
        ok = ok && lapU[s] && Kbu[s] && Kbp[s];
    }
    if (ok) {
        /* forward recomputation of the stage inputs U_s and L U_s */
        memcpy(Yu, u, (size_t)n * sizeof(double));
        memcpy(Yp, pi, (size_t)n * sizeof(double));
        for (int s = 0; s < 4; ++s) {
            oracle_lap_periodic(Yu, lapU[s], nx, ny, nz, h);
            if (s < 3) {
                const double a = RK_A[s + 1] * dt;
                for (i64 i = 0; i < n; ++i) {
                    Ku[i] = Yp[i];
                    Kp[i] = c2[i] * lapU[s][i];
                }
                for (i64 i = 0; i < n; ++i) {
                    Yu[i] = u[i] + a * Ku[i];
                    Yp[i] = pi[i] + a * Kp[i];
                }
            }
        }
        /* reverse sweep over the stages */
        for (int s = 0; s < 4; ++s) {
            const double w = RK_B[s] * dt;
            for (i64 i = 0; i < n; ++i) {
                Kbu[s][i] = w * bu[i];
                Kbp[s][i] = w * bpi[i];
            }
        }
        memcpy(ybu, bu, (size_t)n * sizeof(double));
        memcpy(ybp, bpi, (size_t)n * sizeof(double));
        for (int s = 3; s >= 0; --s) {
            /* Yb_s = A^T Kb_s = ( L(c2 * Kb_s^pi), Kb_s^u ) */
            for (i64 i = 0; i < n; ++i) t[i] = c2[i] * Kbp[s][i];
            oracle_lap_periodic(t, lt, nx, ny, nz, h);
            for (i64 i = 0; i < n; ++i) {
                bc2[i] += Kbp[s][i] * lapU[s][i];
                const double Ybu = lt[i];
                const double Ybp = Kbu[s][i];
                ybu[i] += Ybu;
                ybp[i] += Ybp;
                if (s > 0) {
                    const double a = RK_A[s] * dt;
                    Kbu[s - 1][i] += a * Ybu;
                    Kbp[s - 1][i] += a * Ybp;
                }
            }
        }
        memcpy(bu, ybu, (size_t)n * sizeof(double));
        memcpy(bpi, ybp, (size_t)n * sizeof(double));
    }
    free(Yu); free(Yp); free(Ku); free(Kp); free(t); free(lt); free(ybu); free(ybp);
    for (int s = 0; s < 4; ++s) { free(lapU[s]); free(Kbu[s]); free(Kbp[s]); }
    return ok ? 0 : -1;
}

/*
 * Gradient of a loss of the final state after nsteps RK4 steps, by a
 * checkpointed reverse sweep: the forward run keeps the state every
 * ckpt_every steps; each segment is recomputed forward from its checkpoint,
 * keeping every step's input state, and then reversed step by step.
 *   in:  u0, pi0, c2, (gu_T, gpi_T) = dLoss/d(u_T, pi_T)
 *   out: g_u0, g_pi0 = dLoss/d(u0, pi0);  g_c2 = dLoss/dc2 (overwritten)
 */
int oracle_grad_periodic(const double *u0, const double *pi0, const double *c2,
                         i64 nx, i64 ny, i64 nz, double h, double dt,
                         i64 nsteps, i64 ckpt_every,
                         const double *gu_T, const double *gpi_T,
                         double *g_u0, double *g_pi0, double *g_c2)
{
    const i64 n = nx * ny * nz;
    if (ckpt_every < 1) ckpt_every = 1;
    const i64 nck = (nsteps + ckpt_every - 1) / ckpt_every;
    double *cu = alloc_d((nck > 0 ? nck : 1) * n), *cp = alloc_d((nck > 0 ? nck : 1) * n);
    double *su = alloc_d(ckpt_every * n), *sp = alloc_d(ckpt_every * n);
    double *wu = alloc_d(n), *wp = alloc_d(n);
    int rc = 0;
    if (!(cu && cp && su && sp && wu && wp)) { rc = -1; goto done; }

    /* forward sweep, checkpoint at steps 0, K, 2K, ... */
    memcpy(wu, u0, (size_t)n * sizeof(double));
    memcpy(wp, pi0, (size_t)n * sizeof(double));
    for (i64 c = 0; c < nck; ++c) {
        memcpy(cu + c * n, wu, (size_t)n * sizeof(double));
        memcpy(cp + c * n, wp, (size_t)n * sizeof(double));
        i64 len = nsteps - c * ckpt_every;
        if (len > ckpt_every) len = ckpt_every;
        if (oracle_rk4_periodic(wu, wp, c2, nx, ny, nz, h, dt, len)) { rc = -1; goto done; }
    }

    memcpy(g_u0, gu_T, (size_t)n * sizeof(double));
    memcpy(g_pi0, gpi_T, (size_t)n * sizeof(double));
    memset(g_c2, 0, (size_t)n * sizeof(double));
    for (i64 c = nck - 1; c >= 0; --c) {
        i64 len = nsteps - c * ckpt_every;
        if (len > ckpt_every) len = ckpt_every;
        /* recompute the segment, keeping each step's input state */
        memcpy(wu, cu + c * n, (size_t)n * sizeof(double));
        memcpy(wp, cp + c * n, (size_t)n * sizeof(double));
        for (i64 s = 0; s < len; ++s) {
            memcpy(su + s * n, wu, (size_t)n * sizeof(double));
            memcpy(sp + s * n, wp, (size_t)n * sizeof(double));
            if (oracle_rk4_periodic(wu, wp, c2, nx, ny, nz, h, dt, 1)) { rc = -1; goto done; }
        }
        for (i64 s = len - 1; s >= 0; --s)
            if (oracle_adj_step_periodic(su + s * n, sp + s * n, c2, g_u0, g_pi0, g_c2,
                                         nx, ny, nz, h, dt)) { rc = -1; goto done; }
    }
done:
    free(cu); free(cp); free(su); free(sp); free(wu); free(wp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Ghost exchange on a level of boxes, by brute force                         */
/* ------------------------------------------------------------------------ */

/*
 * A level: nboxes boxes, box b = half-open [lo, hi) in integer grid
 * coordinates, boxes[6*b + 0..2] = lo, boxes[6*b + 3..5] = hi, all inside
 * one domain dom[0..2] = lo, dom[3..5] = hi, periodic along axis d when bit
 * d of periodic is set.  The ghost region of a box is the star-shaped set of
 * points within 2 of a face along exactly one axis (the points the stencil
 * reads).  Edge and corner points of the padded box are not ghosts.
 *
 * The owner of a ghost point p is the unique box o and interior point q of
 * o with q == p after wrapping the periodic axes into the domain.  A ghost
 * with no owner (outside a non-periodic face) has none and is skipped.
 */
static int find_owner(int nboxes, const i64 *boxes, const i64 *dom, int periodic,
                      const i64 p[3], i64 q[3])
{
    for (int d = 0; d < 3; ++d) {
        const i64 len = dom[3 + d] - dom[d];
        if (periodic & (1 << d))
            q[d] = dom[d] + wrap(p[d] - dom[d], len);
        else
            q[d] = p[d];
        if (q[d] < dom[d] || q[d] >= dom[3 + d]) return -1;
    }
    int found = -1;
    for (int o = 0; o < nboxes; ++o) {
        const i64 *B = boxes + 6 * o;
        if (q[0] >= B[0] && q[0] < B[3] && q[1] >= B[1] && q[1] < B[4] &&
            q[2] >= B[2] && q[2] < B[5]) {
            if (found >= 0) return -2; /* overlapping boxes: not a level */
            found = o;
        }
    }
    return found;
}

/* Visit every star ghost point p of box b in a fixed order; call fn. */
typedef void (*ghost_fn)(void *ctx, int b, const i64 p[3]);

static void for_each_ghost(const i64 *B, int b, ghost_fn fn, void *ctx)
{
    for (int d = 0; d < 3; ++d) {
        for (int side = 0; side < 2; ++side) {
            i64 lo[3] = {B[0], B[1], B[2]}, hi[3] = {B[3], B[4], B[5]};
            if (side == 0) { hi[d] = B[d]; lo[d] = B[d] - 2; }
            else { lo[d] = B[3 + d]; hi[d] = B[3 + d] + 2; }
            i64 p[3];
            for (p[2] = lo[2]; p[2] < hi[2]; ++p[2])
                for (p[1] = lo[1]; p[1] < hi[1]; ++p[1])
                    for (p[0] = lo[0]; p[0] < hi[0]; ++p[0])
                        fn(ctx, b, p);
        }
    }
}

struct fill_ctx {
    int nboxes; const i64 *boxes; const i64 *dom; int periodic;
    double **fields; int err;
};

/* offset of grid point p inside box o's dense padded array */
static i64 padded_index(const i64 *B, const i64 p[3])
{
    const i64 px = B[3] - B[0] + 4, py = B[4] - B[1] + 4;
    return ((p[2] - B[2] + 2) * py + (p[1] - B[1] + 2)) * px + (p[0] - B[0] + 2);
}

static void fill_one(void *vctx, int b, const i64 p[3])
{
    struct fill_ctx *c = (struct fill_ctx *)vctx;
    i64 q[3];
    int o = find_owner(c->nboxes, c->boxes, c->dom, c->periodic, p, q);
    if (o == -2) { c->err = -2; return; }
    if (o < 0) return;
    c->fields[b][padded_index(c->boxes + 6 * b, p)] =
        c->fields[o][padded_index(c->boxes + 6 * o, q)];
}

/*
 * Fill the ghost points of every box of one domain.  fields[b] is box b's
 * dense padded array, (nz+4)*(ny+4)*(nx+4) doubles, x fastest.
 * Returns 0, or -2 if two boxes overlap.
 */
int oracle_fill_ghosts(int nboxes, const i64 *boxes, const i64 *dom, int periodic,
                       double **fields)
{
    struct fill_ctx c = {nboxes, boxes, dom, periodic, fields, 0};
    for (int b = 0; b < nboxes; ++b)
        for_each_ghost(boxes + 6 * b, b, fill_one, &c);
    return c.err;
}

struct owner_ctx {
    int nboxes; const i64 *boxes; const i64 *dom; int periodic;
    i64 *out; i64 cap; i64 n; int err;
};

static void owner_one(void *vctx, int b, const i64 p[3])
{
    struct owner_ctx *c = (struct owner_ctx *)vctx;
    i64 q[3];
    int o = find_owner(c->nboxes, c->boxes, c->dom, c->periodic, p, q);
    if (o == -2) { c->err = -2; return; }
    if (o < 0) return;
    if (c->n < c->cap) {
        i64 *r = c->out + 8 * c->n;
        r[0] = b; r[1] = p[0]; r[2] = p[1]; r[3] = p[2];
        r[4] = o; r[5] = q[0]; r[6] = q[1]; r[7] = q[2];
    }
    c->n++;
}

/*
 * The ghost exchange as an explicit point map: one row
 * (dst_box, px, py, pz, src_box, qx, qy, qz) per owned ghost point, in grid
 * coordinates.  Writes at most cap rows; returns the total number of rows
 * (call with cap = 0 to size the buffer), or -2 if two boxes overlap.
 */
i64 oracle_ghost_owners(int nboxes, const i64 *boxes, const i64 *dom, int periodic,
                        i64 *out, i64 cap)
{
    struct owner_ctx c = {nboxes, boxes, dom, periodic, out, cap, 0, 0};
    for (int b = 0; b < nboxes; ++b)
        for_each_ghost(boxes + 6 * b, b, owner_one, &c);
    return c.err ? c.err : c.n;
}
