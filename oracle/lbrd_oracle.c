/*
 * Plain FP64 CPU oracle of the lattice-Boltzmann reaction-diffusion step of
 * Ayodele, Varnik and Raabe, "Lattice Boltzmann study of pattern formation in
 * reaction-diffusion systems" (arXiv 1007.3109).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  It shares no source, header,
 * table or helper with the CUDA library; only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  The product path
 * never calls into it.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fopenmp -fPIC -shared
 *        (no FMA contraction, no fast-math: every operation is one IEEE
 *        double rounding, in the order written below).
 *
 * State layout: f[s][i][y][x], x fastest, one double per value.  The oracle
 * keeps the PRE-collision distributions f_i,s(x, t) of the paper and applies
 * the LB equation literally as a push: the post-collision value computed at
 * site x is written to site x + e_i (periodic).
 *
 * Method (Sec. II.A):
 *   Eq. relax (multi-species form) / Eq. app1 with dt = 1:
 *     f_i,s(x + e_i, t + 1) = f_i,s(x, t)
 *                             + (f_i,s^eq(x, t) - f_i,s(x, t)) / tau_s
 *                             + w_i R_s
 *   Eq. equili:  f_i,s^eq = w_i rho_s   (zero solvent velocity)
 *   rho_s = sum_i f_i,s                 (the moment below Eq. relax)
 *   Eq. Weights: D2Q9 weights 4/9, 1/9, 1/36.
 * Readings where the paper is silent:
 *   - "/ tau_s" is applied as "* omega_s" with omega_s = 1 / tau_s computed
 *     once per species (the two differ only in the last bit).
 *   - velocity order e = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
 *     (-1,-1),(1,-1); rho is summed in that index order.
 *   - D2Q5 (not in the paper): w_0 = 1/3, w_1..4 = 1/6, same c_s^2 = 1/3.
 *   - R_s is evaluated from the pre-collision densities of the same site and
 *     time step.
 * Reactions:
 *   kind 1, transformation A -> B at rate kappa (Sec. II.B, Eq. reac_diff2,
 *     Eq. reac_diff3): R_A = -kappa rho_A, and for a second species
 *     R_B = +kappa rho_A.
 *   kind 2, Gray-Scott (Sec. III, Eq. reac_diff10 / reac_diff11) in Pearson's
 *     lattice form with A0 = k1 = 1, k_f = F, k_0 = k_f, k_2 = k, u = A, v = B:
 *     R_u = -u v^2 + F (1 - u),  R_v = u v^2 - (F + k) v.
 *   kind 3, a mass-action network of up to ORC_MAX_R reaction steps among
 *     S <= ORC_MAX_S species (Eq. reac_diff1 is written for N species; the
 *     paper's own systems are built from such steps, e.g. U + 2V -> 3V):
 *     step r proceeds at rate_r = k_r prod_j rho_j^a_rj and changes species
 *     s by nu_rs per event, so R_s = sum_r nu_rs rate_r.  Evaluated as
 *     p = k_r, then p = p * rho_j repeated a_rj times for j = 0 .. S-1, then
 *     R_s = R_s + nu_rs * p for every s with nu_rs != 0, reactions in order.
 */
#include <stddef.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_MAX_S 4
#define ORC_MAX_R 16

/* A reaction source: kind 0..2 with (kappa, F, k), or kind 3 with a network
 * (order[r][s] = a_rs >= 0, change[r][s] = nu_rs). */
typedef struct {
    int kind;
    double kappa, F, k;
    int nr;
    double rate[ORC_MAX_R];
    int order[ORC_MAX_R][ORC_MAX_S];
    int change[ORC_MAX_R][ORC_MAX_S];
} orc_source;

/* Velocity sets and weights (Eq. Weights for D2Q9; D2Q5 by the reading
 * above).  Returns Q, or 0 for an unknown lattice. */
int orc_lattice(int lattice, int *ex, int *ey, double *w)
{
    static const int ex9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int ey9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    static const int ex5[5] = {0, 1, 0, -1, 0};
    static const int ey5[5] = {0, 0, 1, 0, -1};
    int q;
    if (lattice == 0) {
        for (q = 0; q < 9; ++q) {
            ex[q] = ex9[q];
            ey[q] = ey9[q];
            if (q == 0)
                w[q] = 4.0 / 9.0;
            else if (q <= 4)
                w[q] = 1.0 / 9.0;
            else
                w[q] = 1.0 / 36.0;
        }
        return 9;
    }
    if (lattice == 1) {
        for (q = 0; q < 5; ++q) {
            ex[q] = ex5[q];
            ey[q] = ey5[q];
            w[q] = (q == 0) ? 1.0 / 3.0 : 1.0 / 6.0;
        }
        return 5;
    }
    return 0;
}

/* Reaction source R_s of one site from its densities rho[0..S-1]. */
void orc_reaction(int kind, double kappa, double F, double k, int S,
                  const double *rho, double *R)
{
    int s;
    for (s = 0; s < S; ++s)
        R[s] = 0.0;
    if (kind == 1) {
        R[0] = -kappa * rho[0];
        if (S == 2)
            R[1] = kappa * rho[0];
    } else if (kind == 2 && S == 2) {
        double u = rho[0];
        double v = rho[1];
        double uvv = u * v * v;
        R[0] = -uvv + F * (1.0 - u);
        R[1] = uvv - (F + k) * v;
    }
}

/* Mass-action source of one site (kind 3, see the header). */
static void network_reaction(const orc_source *src, int S, const double *rho, double *R)
{
    int r, j, e, s;
    for (s = 0; s < S; ++s)
        R[s] = 0.0;
    for (r = 0; r < src->nr; ++r) {
        double p = src->rate[r];
        for (j = 0; j < S; ++j)
            for (e = 0; e < src->order[r][j]; ++e)
                p = p * rho[j];
        for (s = 0; s < S; ++s)
            if (src->change[r][s] != 0)
                R[s] = R[s] + (double)src->change[r][s] * p;
    }
}

static void source_eval(const orc_source *src, int S, const double *rho, double *R)
{
    if (src->kind == 3)
        network_reaction(src, S, rho, R);
    else
        orc_reaction(src->kind, src->kappa, src->F, src->k, S, rho, R);
}

/* R of one site under a network given as flat arrays (rate[nr],
 * order[nr * S], change[nr * S], row r = reaction step). */
int orc_network_reaction(int S, int nr, const double *rate, const int *order, const int *change,
                         const double *rho, double *R)
{
    orc_source src;
    int r, s;
    if (S < 1 || S > ORC_MAX_S || nr < 0 || nr > ORC_MAX_R)
        return ORC_EINVAL;
    src.kind = 3;
    src.nr = nr;
    for (r = 0; r < nr; ++r) {
        src.rate[r] = rate[r];
        for (s = 0; s < S; ++s) {
            src.order[r][s] = order[r * S + s];
            src.change[r][s] = change[r * S + s];
        }
    }
    network_reaction(&src, S, rho, R);
    return ORC_OK;
}

static int check_args(int lattice, int S, int64_t nx, int64_t ny, int kind)
{
    if (lattice != 0 && lattice != 1)
        return ORC_EINVAL;
    if (S < 1 || S > ORC_MAX_S || nx < 1 || ny < 1)
        return ORC_EINVAL;
    if (kind < 0 || kind > 3 || (kind == 2 && S != 2) || (kind == 1 && S > 2))
        return ORC_EINVAL;
    return ORC_OK;
}

static size_t at(int64_t nx, int64_t ny, int Q, int s, int i, int64_t y, int64_t x)
{
    return (((size_t)s * (size_t)Q + (size_t)i) * (size_t)ny + (size_t)y) * (size_t)nx + (size_t)x;
}

/* Initial state at equilibrium with the given densities:
 * f_i,s(x, 0) = w_i rho0_s(x)  (Eq. equili; the paper does not state the
 * initial distributions, equilibrium is the reading taken). */
int orc_init(int lattice, int S, int64_t nx, int64_t ny, const double *rho0, double *f)
{
    int ex[9], ey[9];
    double w[9];
    int Q, s, i;
    int64_t y, x;
    if (check_args(lattice, S, nx, ny, 0))
        return ORC_EINVAL;
    Q = orc_lattice(lattice, ex, ey, w);
    for (s = 0; s < S; ++s)
        for (i = 0; i < Q; ++i)
            for (y = 0; y < ny; ++y)
                for (x = 0; x < nx; ++x)
                    f[at(nx, ny, Q, s, i, y, x)] = w[i] * rho0[((size_t)s * ny + y) * nx + x];
    return ORC_OK;
}

/* Densities rho_s(x, t) = sum_i f_i,s(x, t), summed in index order. */
int orc_density(int lattice, int S, int64_t nx, int64_t ny, const double *f, double *rho)
{
    int ex[9], ey[9];
    double w[9];
    int Q, s, i;
    int64_t y, x;
    if (check_args(lattice, S, nx, ny, 0))
        return ORC_EINVAL;
    Q = orc_lattice(lattice, ex, ey, w);
    for (s = 0; s < S; ++s)
        for (y = 0; y < ny; ++y)
            for (x = 0; x < nx; ++x) {
                double r = 0.0;
                for (i = 0; i < Q; ++i)
                    r += f[at(nx, ny, Q, s, i, y, x)];
                rho[((size_t)s * ny + y) * nx + x] = r;
            }
    return ORC_OK;
}

/* One time step t -> t+1: collide every site, then push each post-collision
 * value to its neighbour x + e_i with periodic wrap in x and y (periodic
 * boundaries as in Sec. II.B and Sec. IV).  f_in and f_out must not alias. */
static int step_impl(int lattice, int S, int64_t nx, int64_t ny, const double *tau, const orc_source *src,
                     const double *f_in, double *f_out)
{
    int ex[9], ey[9];
    double w[9];
    double omega[ORC_MAX_S];
    int Q, s;
    int64_t y;
    if (check_args(lattice, S, nx, ny, src->kind))
        return ORC_EINVAL;
    for (s = 0; s < S; ++s) {
        if (!(tau[s] > 0.5))
            return ORC_EINVAL;
        omega[s] = 1.0 / tau[s];
    }
    Q = orc_lattice(lattice, ex, ey, w);
#pragma omp parallel for schedule(static)
    for (y = 0; y < ny; ++y) {
        int64_t x;
        for (x = 0; x < nx; ++x) {
            double rho[ORC_MAX_S], R[ORC_MAX_S];
            int ss, i;
            for (ss = 0; ss < S; ++ss) {
                double r = 0.0;
                for (i = 0; i < Q; ++i)
                    r += f_in[at(nx, ny, Q, ss, i, y, x)];
                rho[ss] = r;
            }
            source_eval(src, S, rho, R);
            for (ss = 0; ss < S; ++ss) {
                for (i = 0; i < Q; ++i) {
                    double fi = f_in[at(nx, ny, Q, ss, i, y, x)];
                    double feq = w[i] * rho[ss];
                    double post = fi + (feq - fi) * omega[ss] + w[i] * R[ss];
                    int64_t x2 = (x + ex[i] + nx) % nx;
                    int64_t y2 = (y + ey[i] + ny) % ny;
                    f_out[at(nx, ny, Q, ss, i, y2, x2)] = post;
                }
            }
        }
    }
    return ORC_OK;
}

static orc_source simple_source(int kind, double kappa, double F, double k)
{
    orc_source src;
    src.kind = kind;
    src.kappa = kappa;
    src.F = F;
    src.k = k;
    src.nr = 0;
    return src;
}

int orc_step(int lattice, int S, int64_t nx, int64_t ny, const double *tau,
             int kind, double kappa, double F, double k,
             const double *f_in, double *f_out)
{
    orc_source src = simple_source(kind, kappa, F, k);
    if (kind == 3)
        return ORC_EINVAL;
    return step_impl(lattice, S, nx, ny, tau, &src, f_in, f_out);
}

static int run_impl(int lattice, int S, int64_t nx, int64_t ny, const double *tau, const orc_source *src,
                    int64_t nsteps, double *f, double *tmp)
{
    int64_t t;
    int Q = (lattice == 0) ? 9 : 5;
    size_t n = (size_t)S * (size_t)Q * (size_t)nx * (size_t)ny;
    double *a = f, *b = tmp;
    for (t = 0; t < nsteps; ++t) {
        double *c;
        int rc = step_impl(lattice, S, nx, ny, tau, src, a, b);
        if (rc)
            return rc;
        c = a;
        a = b;
        b = c;
    }
    if (a != f) {
        size_t j;
        for (j = 0; j < n; ++j)
            f[j] = a[j];
    }
    return ORC_OK;
}

/* nsteps steps on f; tmp is a caller buffer of the same size.  The two
 * buffers alternate, and the final state is left in f. */
int orc_run(int lattice, int S, int64_t nx, int64_t ny, const double *tau,
            int kind, double kappa, double F, double k, int64_t nsteps,
            double *f, double *tmp)
{
    orc_source src = simple_source(kind, kappa, F, k);
    if (kind == 3)
        return ORC_EINVAL;
    return run_impl(lattice, S, nx, ny, tau, &src, nsteps, f, tmp);
}

/* orc_run with a mass-action network (kind 3) given as flat arrays as in
 * orc_network_reaction. */
int orc_run_network(int lattice, int S, int64_t nx, int64_t ny, const double *tau,
                    int nr, const double *rate, const int *order, const int *change, int64_t nsteps,
                    double *f, double *tmp)
{
    orc_source src = simple_source(3, 0.0, 0.0, 0.0);
    int r, s;
    if (S < 1 || S > ORC_MAX_S || nr < 0 || nr > ORC_MAX_R)
        return ORC_EINVAL;
    src.nr = nr;
    for (r = 0; r < nr; ++r) {
        src.rate[r] = rate[r];
        for (s = 0; s < S; ++s) {
            src.order[r][s] = order[r * S + s];
            src.change[r][s] = change[r * S + s];
        }
    }
    return run_impl(lattice, S, nx, ny, tau, &src, nsteps, f, tmp);
}

/* Set the number of threads of the parallel loops (n >= 1); returns it. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Number of threads the parallel loops use. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
