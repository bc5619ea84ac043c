/*
 * Plain FP64 CPU oracle for softened direct-summation gravity.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark do. It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Every routine is the definition written out, slowly and plainly:
 *   - inputs are FP32 particle records (x, y, z, m) widened exactly to FP64
 *     (the j-particle record of the paper's appendix driver: JDIM = 4), and
 *     the softening eps2 is the FP32 value widened the same way;
 *   - each sum runs over j in ascending order in FP64 with Neumaier
 *     compensation, so its result is the exact sum to about 1 ulp of FP64;
 *   - OpenMP splits only the independent i rows; each row's arithmetic is
 *     sequential and identical for any thread count.
 *
 * Readings of points the paper leaves open (also listed in the design
 * notes):
 *   - G = 1; r_ij = r_j - r_i (Section 1.1, Eq. 1).
 *   - eps2 is eps^2, added to r^2 before the inverse square root (the force
 *     pipeline description of the appendix adds eps2 to dx^2 + dy^2 + dz^2).
 *   - a pair whose softened distance s = r^2 + eps2 is exactly 0 (only
 *     possible with eps2 = 0 and coincident points) contributes nothing.
 *   - the potential phi_i = -sum_j m_j / sqrt(r_ij^2 + eps2) (sign from the
 *     force-jerk-potential pipeline description of the appendix, which
 *     subtracts the pair potential from its output) skips every pair whose
 *     separation is exactly zero, which removes the i = j self term.
 *
 * Parity pins: every function here is checked by the CPU test suite
 * against closed forms, conservation laws, finite differences and a
 * 50-digit brute force; none is "parity unpinned".
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Neumaier (improved Kahan) compensated sum. */
typedef struct {
    double s;
    double c;
} nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_value(const nsum *a) { return a->s + a->c; }

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Eq. 1 of Section 1.1 (acceleration) plus the potential for one i-particle
 * at (xi, yi, zi) with softening eps2:
 *   a_i   =  sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps2)^(3/2)
 *   phi_i = -sum_{j : x_j != x_i} m_j / (|x_j - x_i|^2 + eps2)^(1/2)
 * out[0..2] = a_i, out[3] = phi_i (when want_pot).
 */
static void force_row(double xi, double yi, double zi, double eps2, int64_t n_j, const float *pos_mass_j,
                      int want_pot, double out[4])
{
    nsum ax = {0, 0}, ay = {0, 0}, az = {0, 0}, ph = {0, 0};
    for (int64_t j = 0; j < n_j; ++j) {
        const double dx = (double)pos_mass_j[4 * j + 0] - xi;
        const double dy = (double)pos_mass_j[4 * j + 1] - yi;
        const double dz = (double)pos_mass_j[4 * j + 2] - zi;
        const double mj = pos_mass_j[4 * j + 3];
        const double s = dx * dx + dy * dy + dz * dz + eps2;
        if (s == 0.0)
            continue;
        const double root = sqrt(s);
        const double f = mj / (s * root); /* m_j / s^(3/2) */
        nsum_add(&ax, f * dx);
        nsum_add(&ay, f * dy);
        nsum_add(&az, f * dz);
        if (want_pot && !(dx == 0.0 && dy == 0.0 && dz == 0.0))
            nsum_add(&ph, -mj / root);
    }
    out[0] = nsum_value(&ax);
    out[1] = nsum_value(&ay);
    out[2] = nsum_value(&az);
    out[3] = nsum_value(&ph);
}

/*
 * Eq. 1 for the listed i-particles with one softening for all pairs.
 * rows: indices of the i-particles to evaluate (NULL means 0 .. n_rows-1).
 * pos_i: FP32 [*, 4] records (the 4th component is ignored).
 * pos_mass_j: FP32 [n_j, 4] records (x, y, z, m).
 * acc: FP64 [n_rows, 3] output (row order of `rows`); pot: FP64 [n_rows] or NULL.
 */
void oracle_force_rows(int64_t n_rows, const int64_t *rows, const float *pos_i,
                       int64_t n_j, const float *pos_mass_j, float eps2_f,
                       double *acc, double *pot)
{
    const double eps2 = (double)eps2_f;
    int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < n_rows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        double out[4];
        force_row(pos_i[4 * i + 0], pos_i[4 * i + 1], pos_i[4 * i + 2], eps2, n_j, pos_mass_j, pot != NULL, out);
        acc[3 * r + 0] = out[0];
        acc[3 * r + 1] = out[1];
        acc[3 * r + 2] = out[2];
        if (pot)
            pot[r] = out[3];
    }
}

/*
 * Eq. 1 with a softening per i-particle: the i record of the appendix's
 * force driver is (x, y, z, eps2) (IDIM = 4, the driver fills the 4th slot
 * with eps2), and the force pipeline adds that i-particle's eps2 to the
 * squared distance of each of its pairs. pos_eps_i: FP32 [*, 4] records
 * (x, y, z, eps2_i); everything else as oracle_force_rows.
 */
void oracle_force_rows_eps_i(int64_t n_rows, const int64_t *rows, const float *pos_eps_i,
                             int64_t n_j, const float *pos_mass_j, double *acc, double *pot)
{
    int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < n_rows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        double out[4];
        force_row(pos_eps_i[4 * i + 0], pos_eps_i[4 * i + 1], pos_eps_i[4 * i + 2], (double)pos_eps_i[4 * i + 3],
                  n_j, pos_mass_j, pot != NULL, out);
        acc[3 * r + 0] = out[0];
        acc[3 * r + 1] = out[1];
        acc[3 * r + 2] = out[2];
        if (pot)
            pot[r] = out[3];
    }
}

/*
 * Acceleration, its time derivative (jerk) and the potential - the outputs
 * of the force-jerk-potential pipeline description of the appendix - for
 * particles moving with velocities v:
 *   a_i   =  sum_j m_j d / s^(3/2)
 *   j_i   =  sum_j m_j [ w / s^(3/2) - 3 (d . w) d / s^(5/2) ]
 *   phi_i = -sum_{j : d != 0} m_j / s^(1/2)
 * with d = x_j - x_i, w = v_j - v_i, s = |d|^2 + eps2 (j_i is d a_i / dt
 * for straight-line motion). vel_i, vel_j are FP32 [*, 4] records (the 4th
 * component is ignored). Pairs with s = 0 are skipped.
 */
void oracle_force_jerk_rows(int64_t n_rows, const int64_t *rows, const float *pos_i, const float *vel_i,
                            int64_t n_j, const float *pos_mass_j, const float *vel_j, float eps2_f,
                            double *acc, double *jerk, double *pot)
{
    const double eps2 = (double)eps2_f;
    int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < n_rows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        const double xi = pos_i[4 * i + 0], yi = pos_i[4 * i + 1], zi = pos_i[4 * i + 2];
        const double ui = vel_i[4 * i + 0], vi = vel_i[4 * i + 1], wi = vel_i[4 * i + 2];
        nsum ax = {0, 0}, ay = {0, 0}, az = {0, 0};
        nsum jx = {0, 0}, jy = {0, 0}, jz = {0, 0}, ph = {0, 0};
        for (int64_t j = 0; j < n_j; ++j) {
            const double dx = (double)pos_mass_j[4 * j + 0] - xi;
            const double dy = (double)pos_mass_j[4 * j + 1] - yi;
            const double dz = (double)pos_mass_j[4 * j + 2] - zi;
            const double wx = (double)vel_j[4 * j + 0] - ui;
            const double wy = (double)vel_j[4 * j + 1] - vi;
            const double wz = (double)vel_j[4 * j + 2] - wi;
            const double mj = pos_mass_j[4 * j + 3];
            const double s = dx * dx + dy * dy + dz * dz + eps2;
            if (s == 0.0)
                continue;
            const double root = sqrt(s);
            const double g = mj / (s * root);           /* m / s^(3/2) */
            const double h = 3.0 * (dx * wx + dy * wy + dz * wz) / s;
            nsum_add(&ax, g * dx);
            nsum_add(&ay, g * dy);
            nsum_add(&az, g * dz);
            nsum_add(&jx, g * (wx - h * dx));
            nsum_add(&jy, g * (wy - h * dy));
            nsum_add(&jz, g * (wz - h * dz));
            if (pot && !(dx == 0.0 && dy == 0.0 && dz == 0.0))
                nsum_add(&ph, -mj / root);
        }
        acc[3 * r + 0] = nsum_value(&ax);
        acc[3 * r + 1] = nsum_value(&ay);
        acc[3 * r + 2] = nsum_value(&az);
        jerk[3 * r + 0] = nsum_value(&jx);
        jerk[3 * r + 1] = nsum_value(&jy);
        jerk[3 * r + 2] = nsum_value(&jz);
        if (pot)
            pot[r] = nsum_value(&ph);
    }
}

/* Potential energy W = 1/2 sum_i m_i phi_i (FP64, Neumaier, i ascending). */
double oracle_potential_energy(int64_t n, const float *pos_mass, const double *pot)
{
    nsum w = {0, 0};
    for (int64_t i = 0; i < n; ++i)
        nsum_add(&w, 0.5 * (double)pos_mass[4 * i + 3] * pot[i]);
    return nsum_value(&w);
}

/*
 * Analytic gradient of L = sum_i w_i . a_i with respect to every position
 * and mass (the adjoint pass; the paper has no counterpart, it is the
 * derivative of Eq. 1). With d = x_p - x_k, s = |d|^2 + eps2,
 * g = s^(-3/2), h = s^(-5/2) and u = m_k w_p - m_p w_k:
 *   dL/dx_k = sum_p [ g u - 3 h (d . u) d ]
 *   dL/dm_k = -sum_p g (w_p . d)
 * Derivation: a_i depends on x_k through the i = k terms (sign -1 on d) and
 * the j = k terms (sign +1), and the Jacobian of d s^(-3/2) is
 * g I - 3 h d d^T, which is even in d. The p = k term vanishes (u = 0,
 * d = 0); pairs with s = 0 are skipped as in the force.
 *
 * rows: indices k to evaluate (NULL means all n). grad_pos: FP64 [n_rows,3];
 * grad_mass: FP64 [n_rows] (either may be NULL).
 */
void oracle_adjoint_rows(int64_t n_rows, const int64_t *rows, int64_t n,
                         const float *pos_mass, float eps2_f, const float *w,
                         double *grad_pos, double *grad_mass)
{
    const double eps2 = (double)eps2_f;
    int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < n_rows; ++r) {
        const int64_t k = rows ? rows[r] : r;
        const double xk = pos_mass[4 * k + 0];
        const double yk = pos_mass[4 * k + 1];
        const double zk = pos_mass[4 * k + 2];
        const double mk = pos_mass[4 * k + 3];
        const double wkx = w[3 * k + 0], wky = w[3 * k + 1], wkz = w[3 * k + 2];
        nsum gx = {0, 0}, gy = {0, 0}, gz = {0, 0}, gm = {0, 0};
        for (int64_t p = 0; p < n; ++p) {
            if (p == k)
                continue;
            const double dx = (double)pos_mass[4 * p + 0] - xk;
            const double dy = (double)pos_mass[4 * p + 1] - yk;
            const double dz = (double)pos_mass[4 * p + 2] - zk;
            const double mp = pos_mass[4 * p + 3];
            const double wpx = w[3 * p + 0], wpy = w[3 * p + 1], wpz = w[3 * p + 2];
            const double s = dx * dx + dy * dy + dz * dz + eps2;
            if (s == 0.0)
                continue;
            const double root = sqrt(s);
            const double g = 1.0 / (s * root);
            const double h = g / s;
            const double ux = mk * wpx - mp * wkx;
            const double uy = mk * wpy - mp * wky;
            const double uz = mk * wpz - mp * wkz;
            const double du = dx * ux + dy * uy + dz * uz;
            nsum_add(&gx, g * ux - 3.0 * h * du * dx);
            nsum_add(&gy, g * uy - 3.0 * h * du * dy);
            nsum_add(&gz, g * uz - 3.0 * h * du * dz);
            nsum_add(&gm, -g * (wpx * dx + wpy * dy + wpz * dz));
        }
        if (grad_pos) {
            grad_pos[3 * r + 0] = nsum_value(&gx);
            grad_pos[3 * r + 1] = nsum_value(&gy);
            grad_pos[3 * r + 2] = nsum_value(&gz);
        }
        if (grad_mass)
            grad_mass[r] = nsum_value(&gm);
    }
}

/*
 * The part of L = sum_i w_i . a_i that depends on particle k, with particle
 * k moved to (xk, yk, zk) and given mass mk (FP64 values, so a finite
 * difference can perturb them below FP32 resolution):
 *   L_k = w_k . a_k + sum_{p != k} w_p . [ m_k (x_k - x_p) / s_pk^(3/2) ]
 * Every other term of L is independent of particle k, so central
 * differences of L_k equal central differences of L.
 */
double oracle_loss_k(int64_t n, const float *pos_mass, float eps2_f, const float *w,
                     int64_t k, double xk, double yk, double zk, double mk)
{
    const double eps2 = (double)eps2_f;
    nsum l = {0, 0};
    const double wkx = w[3 * k + 0], wky = w[3 * k + 1], wkz = w[3 * k + 2];
    for (int64_t p = 0; p < n; ++p) {
        if (p == k)
            continue;
        const double dx = (double)pos_mass[4 * p + 0] - xk;
        const double dy = (double)pos_mass[4 * p + 1] - yk;
        const double dz = (double)pos_mass[4 * p + 2] - zk;
        const double mp = pos_mass[4 * p + 3];
        const double s = dx * dx + dy * dy + dz * dz + eps2;
        if (s == 0.0)
            continue;
        const double g = 1.0 / (s * sqrt(s));
        /* w_k . (force of p on k) */
        nsum_add(&l, mp * g * (wkx * dx + wky * dy + wkz * dz));
        /* w_p . (force of k on p): direction x_k - x_p = -d */
        nsum_add(&l, -mk * g * (w[3 * p + 0] * dx + w[3 * p + 1] * dy + w[3 * p + 2] * dz));
    }
    return nsum_value(&l);
}

/*
 * FP32 accumulation study (test-only). Each pair term is formed in IEEE
 * single precision with correctly rounded square root and division, with
 * the softened squared distance grouped as (dx^2 + dy^2) + (dz^2 + eps2)
 * as in the force pipeline description of the appendix, then multiplied
 * by the mass times the cubed inverse distance. The three modes differ
 * only in how the FP32 terms are summed:
 * mode 0: DIRECT style - one FP32 running sum over all j in order
 *         (Section 3.4, the DIRECT column of Table 2).
 * mode 1: FORCE-LOOP - an FP32 "current" sum over each J-BAG of n_jb
 *         j-particles, added into an FP32 "backup" sum after each bag
 *         (Section 2.2.2, Eq. 2).
 * mode 2: the same FP32 pair terms summed exactly (FP64 Neumaier), which
 *         isolates the rounding of the pair arithmetic itself.
 * This file is compiled with -ffp-contract=off, so no multiply-add is fused.
 */
void oracle_fp32_study(int64_t n_rows, const int64_t *rows, const float *pos_i,
                       int64_t n_j, const float *pos_mass_j, float eps2, int mode,
                       int64_t n_jb, double *acc)
{
    int64_t r;
    if (n_jb <= 0)
        n_jb = 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < n_rows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        const float xi = pos_i[4 * i + 0];
        const float yi = pos_i[4 * i + 1];
        const float zi = pos_i[4 * i + 2];
        float bx = 0.f, by = 0.f, bz = 0.f; /* running / backup sum */
        float cx = 0.f, cy = 0.f, cz = 0.f; /* current (per J-BAG) sum */
        nsum ex = {0, 0}, ey = {0, 0}, ez = {0, 0};
        for (int64_t j = 0; j < n_j; ++j) {
            const float ux = pos_mass_j[4 * j + 0] - xi;
            const float uy = pos_mass_j[4 * j + 1] - yi;
            const float uz = pos_mass_j[4 * j + 2] - zi;
            const float mass = pos_mass_j[4 * j + 3];
            const float soft = (ux * ux + uy * uy) + (uz * uz + eps2);
            float fx = 0.f, fy = 0.f, fz = 0.f;
            if (soft != 0.f) {
                const float inv = 1.0f / sqrtf(soft);
                const float coef = mass * ((inv * inv) * inv);
                fx = coef * ux;
                fy = coef * uy;
                fz = coef * uz;
            }
            if (mode == 0) {
                bx += fx;
                by += fy;
                bz += fz;
            } else if (mode == 1) {
                cx += fx;
                cy += fy;
                cz += fz;
                if ((j + 1) % n_jb == 0 || j + 1 == n_j) {
                    bx += cx;
                    by += cy;
                    bz += cz;
                    cx = cy = cz = 0.f;
                }
            } else {
                nsum_add(&ex, (double)fx);
                nsum_add(&ey, (double)fy);
                nsum_add(&ez, (double)fz);
            }
        }
        if (mode == 2) {
            acc[3 * r + 0] = nsum_value(&ex);
            acc[3 * r + 1] = nsum_value(&ey);
            acc[3 * r + 2] = nsum_value(&ez);
        } else {
            acc[3 * r + 0] = bx;
            acc[3 * r + 1] = by;
            acc[3 * r + 2] = bz;
        }
    }
}
