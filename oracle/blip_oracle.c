/*
 * FP64 CPU oracle for the periodic cubic-blip orbital evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (Sec. II.B of Uejima & Maezono, Eqs. 11.12.24.1, 11.12.24.2
 * and 7): for every electron position r_j and every orbital l,
 *
 *     psi_l(r_j) = sum over the 4^3 = 64 grid sites s whose basis function is
 *                  non-zero at r_j of  a_{l,s} * Theta_s(r_j),
 *     Theta_s(r) = phi(g_1 - m_1) phi(g_2 - m_2) phi(g_3 - m_3),
 *
 * with g = diag(n) A^{-1} r the grid coordinates of r (A = matrix whose
 * columns are the lattice vectors; site m sits at r = A diag(n)^{-1} m, so for
 * an orthorhombic cell g_a - m_a = (x_a - X_a) / b_a as in Eq. 11.12.24.2),
 * phi the centred cubic B-spline (the paper's "4 points per direction" needs
 * a cubic; the text's "second order polynomial" is read as a misprint), and
 * the coefficient of site m taken at m mod n (periodic cell).  The gradient
 * and Laplacian follow by the chain rule:
 *     grad_r psi = J^T grad_g psi,   lap_r psi = sum_ab (J J^T)_ab d_a d_b psi,
 *     J = diag(n) A^{-1}.
 * Because phi has support [-2, 2], the 64-term sum equals the full sum over
 * all sites and periodic images; the oracle takes the 64 terms in the natural
 * order (x slowest, z fastest), with no blocking or reordering.
 *
 * Everything is double precision.  Electrons are split over POSIX threads;
 * each electron is computed by exactly one thread, so results do not depend on
 * the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * The centred cubic B-spline and its derivatives, piecewise (Eq. 11.12.24.2,
 * phi read as the cubic B-spline of the blip basis):
 *   B(x)   = 2/3 - x^2 + |x|^3/2       |x| <= 1
 *          = (2 - |x|)^3 / 6           1 <= |x| <= 2
 *          = 0                          otherwise
 *   B'(x)  = -2x + 3 x|x| / 2          |x| <= 1
 *          = -sgn(x) (2 - |x|)^2 / 2   1 <= |x| <= 2
 *   B''(x) = -2 + 3|x|                 |x| <= 1
 *          = 2 - |x|                    1 <= |x| <= 2
 * ------------------------------------------------------------------------- */
double oracle_B(double x)
{
    double ax = fabs(x);
    if (ax <= 1.0) return 2.0 / 3.0 - ax * ax + 0.5 * ax * ax * ax;
    if (ax <= 2.0) { double d = 2.0 - ax; return d * d * d / 6.0; }
    return 0.0;
}

double oracle_dB(double x)
{
    double ax = fabs(x);
    if (ax <= 1.0) return -2.0 * x + 1.5 * x * ax;
    if (ax <= 2.0) { double d = 2.0 - ax; return (x > 0 ? -0.5 : 0.5) * d * d; }
    return 0.0;
}

double oracle_d2B(double x)
{
    double ax = fabs(x);
    if (ax <= 1.0) return -2.0 + 3.0 * ax;
    if (ax <= 2.0) return 2.0 - ax;
    return 0.0;
}

/* ---------------------------------------------------------------------------
 * Cell geometry.  lattice[3*i + c] = component c of lattice vector a_i, so the
 * matrix A with the vectors as columns has A[c][i] = lattice[3*i + c].
 * Outputs (row-major 3x3): Ainv = A^{-1} (adjugate / determinant),
 * J = diag(n) A^{-1}, M = J J^T.  Returns 0, or -1 for a singular cell.
 * ------------------------------------------------------------------------- */
int oracle_geometry(const int grid[3], const double lattice[9],
                    double Ainv[9], double J[9], double M[9])
{
    double A[3][3];
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < 3; ++i) A[c][i] = lattice[3 * i + c];
    double cof[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            int r1 = (r + 1) % 3, r2 = (r + 2) % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
            cof[r][c] = A[r1][c1] * A[r2][c2] - A[r1][c2] * A[r2][c1];
        }
    double det = A[0][0] * cof[0][0] + A[0][1] * cof[0][1] + A[0][2] * cof[0][2];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return -1;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ainv[3 * r + c] = cof[c][r] / det;  /* adj = cof^T */
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) J[3 * a + c] = (double)grid[a] * Ainv[3 * a + c];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += J[3 * a + c] * J[3 * b + c];
            M[3 * a + b] = s;
        }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Stencil selection for one axis (Eq. 7: the 4 sites per direction whose
 * basis functions are non-zero at r).  Input: fractional coordinate u (any
 * real).  Output: base index i in [0, n), offset t = g - floor(g) in [0, 1).
 * The wrap u <- u - floor(u) can round up to exactly 1.0 for tiny negative u;
 * that point is the cell origin, so it is mapped to 0.
 * ------------------------------------------------------------------------- */
static void oracle_axis(double u, int n, int *i_out, double *t_out)
{
    double w = u - floor(u);
    if (w >= 1.0) w = 0.0;
    double g = (double)n * w;
    double fi = floor(g);
    double t = g - fi;
    long i = (long)fi % n;
    if (i < 0) i += n;
    *i_out = (int)i;
    *t_out = t;
}

typedef struct {
    int grid[3];
    double Ainv[9], J[9], M[9];
    double norm;               /* 1, or (3/2)^3 for phi(0) = 1 blips */
    int n_orb;
    const double *coeffs;      /* [n1][n2][n3][n_orb] */
    const double *pos;         /* [E][3] */
    double *values;            /* [E][n_orb] */
    double *grads;             /* [E][3][n_orb] */
    double *laps;              /* [E][n_orb] */
    double *absmag;            /* optional [E][5][n_orb]: sum_s |W_k(s)| |a_ls| */
    long e0, e1;
} oracle_job;

static void oracle_one(const oracle_job *jb, long e, double *acc5)
{
    const int n1 = jb->grid[0], n2 = jb->grid[1], n3 = jb->grid[2];
    const int L = jb->n_orb;
    const double *r = jb->pos + 3 * e;

    double *val = jb->values + (size_t)e * L;
    double *grd = jb->grads + (size_t)e * 3 * L;
    double *lap = jb->laps + (size_t)e * L;
    double *mag = jb->absmag ? jb->absmag + (size_t)e * 5 * L : NULL;

    int base[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double u = jb->Ainv[3 * a + 0] * r[0] + jb->Ainv[3 * a + 1] * r[1]
                 + jb->Ainv[3 * a + 2] * r[2];
        if (!isfinite(u)) {           /* no cell for this position: NaN out */
            for (int l = 0; l < L; ++l) {
                val[l] = lap[l] = NAN;
                grd[l] = grd[L + l] = grd[2 * L + l] = NAN;
            }
            if (mag) for (int l = 0; l < 5 * L; ++l) mag[l] = NAN;
            return;
        }
        oracle_axis(u, jb->grid[a], &base[a], &t[a]);
    }

    /* 1-D values: site m = i - 1 + k sits at grid distance g - m = t + 1 - k. */
    double b0[3][4], b1[3][4], b2[3][4];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 4; ++k) {
            double x = t[a] + 1.0 - (double)k;
            b0[a][k] = oracle_B(x);
            b1[a][k] = oracle_dB(x);
            b2[a][k] = oracle_d2B(x);
        }

    memset(acc5, 0, sizeof(double) * 5 * L * 2);
    double *acc = acc5, *accm = acc5 + 5 * L;

    for (int kx = 0; kx < 4; ++kx)
        for (int ky = 0; ky < 4; ++ky)
            for (int kz = 0; kz < 4; ++kz) {
                /* Theta and its derivatives with respect to the grid coordinates */
                double th = b0[0][kx] * b0[1][ky] * b0[2][kz];
                double dg[3] = {b1[0][kx] * b0[1][ky] * b0[2][kz],
                                b0[0][kx] * b1[1][ky] * b0[2][kz],
                                b0[0][kx] * b0[1][ky] * b1[2][kz]};
                double hg[3][3];
                hg[0][0] = b2[0][kx] * b0[1][ky] * b0[2][kz];
                hg[1][1] = b0[0][kx] * b2[1][ky] * b0[2][kz];
                hg[2][2] = b0[0][kx] * b0[1][ky] * b2[2][kz];
                hg[0][1] = hg[1][0] = b1[0][kx] * b1[1][ky] * b0[2][kz];
                hg[0][2] = hg[2][0] = b1[0][kx] * b0[1][ky] * b1[2][kz];
                hg[1][2] = hg[2][1] = b0[0][kx] * b1[1][ky] * b1[2][kz];
                /* chain rule to Cartesian: grad_c = sum_a J_ac dg_a; lap = sum_ab M_ab hg_ab */
                double W[5];
                W[0] = th;
                for (int c = 0; c < 3; ++c)
                    W[1 + c] = jb->J[0 + c] * dg[0] + jb->J[3 + c] * dg[1] + jb->J[6 + c] * dg[2];
                double lp = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) lp += jb->M[3 * a + b] * hg[a][b];
                W[4] = lp;
                for (int k = 0; k < 5; ++k) W[k] *= jb->norm;

                /* coefficient of site m, taken periodically (m mod n) */
                int sx = (base[0] - 1 + kx + n1) % n1;
                int sy = (base[1] - 1 + ky + n2) % n2;
                int sz = (base[2] - 1 + kz + n3) % n3;
                const double *c = jb->coeffs + (((size_t)sx * n2 + sy) * n3 + sz) * (size_t)L;
                for (int k = 0; k < 5; ++k) {
                    double w = W[k], aw = fabs(W[k]);
                    double *ak = acc + (size_t)k * L, *am = accm + (size_t)k * L;
                    for (int l = 0; l < L; ++l) {
                        ak[l] += w * c[l];
                        am[l] += aw * fabs(c[l]);
                    }
                }
            }
    for (int l = 0; l < L; ++l) {
        val[l] = acc[l];
        grd[l] = acc[L + l];
        grd[L + l] = acc[2 * L + l];
        grd[2 * L + l] = acc[3 * L + l];
        lap[l] = acc[4 * L + l];
    }
    if (mag) memcpy(mag, accm, sizeof(double) * 5 * L);
}

static void *oracle_worker(void *arg)
{
    oracle_job *jb = (oracle_job *)arg;
    double *acc = (double *)malloc(sizeof(double) * 10 * (size_t)jb->n_orb);
    if (!acc) return (void *)1;
    for (long e = jb->e0; e < jb->e1; ++e) oracle_one(jb, e, acc);
    free(acc);
    return NULL;
}

/*
 * Evaluate values, gradients and Laplacians of all orbitals at all positions.
 *   grid[3]        grid points along lattice vectors a_1, a_2, a_3
 *   lattice[9]     row i = lattice vector a_i (bohr)
 *   n_orb          real orbitals per grid row (a complex table passes its
 *                  interleaved real/imaginary parts as 2 x n_orb real ones;
 *                  the weights are real, so both parts contract identically)
 *   norm_kind      0: B-spline (partition of unity); 1: phi(0) = 1 blips,
 *                  i.e. every 1-D factor times 3/2
 *   coeffs         [n1][n2][n3][n_orb]
 *   pos            [n_elec][3] Cartesian positions (any real values)
 *   values/grads/laps  [n_elec][n_orb], [n_elec][3][n_orb], [n_elec][n_orb]
 *   absmag         NULL or [n_elec][5][n_orb]: sum_s |W_k(s)| |a_ls| for
 *                  k = value, grad x, y, z, Laplacian (the rounding scale of
 *                  each output)
 *   n_threads      worker threads (<= 0: one)
 * Returns 0, -1 for invalid arguments, -2 for a singular cell, -3 on
 * allocation failure.
 */
int oracle_eval(const int grid[3], const double lattice[9], int n_orb, int norm_kind,
                const double *coeffs, const double *pos, long n_elec,
                double *values, double *grads, double *laps, double *absmag,
                int n_threads)
{
    if (!grid || !lattice || !coeffs || (!pos && n_elec > 0) || n_orb <= 0 || n_elec < 0)
        return -1;
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1) return -1;
    oracle_job base;
    memset(&base, 0, sizeof(base));
    memcpy(base.grid, grid, sizeof(base.grid));
    if (oracle_geometry(grid, lattice, base.Ainv, base.J, base.M) != 0) return -2;
    base.norm = norm_kind == 1 ? 1.5 * 1.5 * 1.5 : 1.0;
    base.n_orb = n_orb;
    base.coeffs = coeffs;
    base.pos = pos;
    base.values = values;
    base.grads = grads;
    base.laps = laps;
    base.absmag = absmag;
    if (n_elec == 0) return 0;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_elec) n_threads = (int)n_elec;

    oracle_job *jobs = (oracle_job *)calloc((size_t)n_threads, sizeof(oracle_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -3; }
    int rc = 0;
    for (int i = 0; i < n_threads; ++i) {
        jobs[i] = base;
        jobs[i].e0 = n_elec * i / n_threads;
        jobs[i].e1 = n_elec * (i + 1) / n_threads;
    }
    char *running = (char *)calloc((size_t)n_threads, 1);
    if (!running) { free(jobs); free(th); return -3; }
    for (int i = 1; i < n_threads; ++i)
        running[i] = pthread_create(&th[i], NULL, oracle_worker, &jobs[i]) == 0;
    if (oracle_worker(&jobs[0]) != NULL) rc = -3;
    for (int i = 1; i < n_threads; ++i) {
        void *ret = NULL;
        if (running[i]) pthread_join(th[i], &ret);
        else ret = oracle_worker(&jobs[i]);   /* no thread: run it here */
        if (ret != NULL) rc = -3;
    }
    free(running);
    free(jobs);
    free(th);
    return rc;
}
