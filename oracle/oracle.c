/*
 * FP64 CPU oracle for square root bundle adjustment (test infrastructure).
 *
 * This file is the plain, slow, obviously-correct reference that the CUDA
 * path is checked against.  It is NOT part of the product: only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It
 * shares no code with the CUDA library.
 *
 * Square root BA reaches, up to rounding, exactly the Schur-complement (SC)
 * result (Sec. 4.4, Eq. red_H / red_b and the back-substitution identity),
 * so the oracle is the plain definition written out:
 *   - energy E = sum ||r_ij||^2                         (Sec. 4, Eq. ba_energy)
 *   - damped linearised problem, D^2 = diag(J^T J)      (Sec. 4.1, Eq. linearized_residual)
 *   - normal equations H, b                             (Sec. 4.1, Eq. normal_eq)
 *   - Schur complement RCS and back substitution        (Sec. 4.2, Eq. red_normal_eq, backsub_sc)
 *     with the damped H_pp + lambda D_p^2, H_ll + lambda D_l^2 (remark closing Sec. 4.4)
 *   - RCS solved densely (Cholesky) or by block-Jacobi PCG (Sec. 5.4, 6.1)
 *   - Levenberg-Marquardt loop: lambda0 = 1e-4, <= 50 iterations, relative
 *     function tolerance 1e-6, <= 500 CG iterations (Sec. 6.1)
 *
 * Readings where the paper is silent (shared with the CUDA path by
 * specification, never by code):
 *   camera: BAL "Snavely" model (Sec. 6.2): P = R(w) X + t, p = -P_xy / P_z,
 *     pixel = f (1 + k1 |p|^2 + k2 |p|^4) p, residual = pixel - z.
 *   rotation increment: left-multiplicative R <- Exp(dw) R, so dP/d(dw) = -[R X]_x;
 *     the composed rotation is stored back as axis-angle via unit quaternions.
 *   D^2 = clamp(diag(J^T J), 1e-6, 1e32) of the unscaled Jacobian (equivalent
 *     to unit column scaling with D = I in exact arithmetic).
 *   lambda update: Nielsen's rule; accept iff rho > 1e-3, the model decrease
 *     E - L is positive and the new cost is finite.
 *     rho = (E - E_new) / (E - L), L = ||r + J dx||^2 (undamped model).
 *   robust norm (Huber, Sec. 6.2, as IRLS; off unless orc_set_huber(delta > 0)):
 *     rho(s) = s for s <= delta^2, 2 delta sqrt(s) - delta^2 above, s = ||r_ij||^2;
 *     E = sum rho(s); the linearised rows [J | r] of an observation are scaled
 *     by sqrt(w), w = rho'(s) = min(1, delta / ||r||); the model of the robust
 *     cost is L = sum rho(s) - w ||r||^2 + w ||r + J dx||^2, so that
 *     E - L = sum w (||r||^2 - ||r + J dx||^2).
 *   CG stop: Nash-Sofer truncated-Newton test i (Q_i - Q_{i-1}) / Q_i < eta with
 *     Q(x) = 1/2 x^T H x - g^T x evaluated as -1/2 x^T (g + r); or ||r|| <= 1e-10 ||g||;
 *     or the iteration limit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads (OpenMP, when built with it): the independent per-observation
 * and per-landmark loops run in parallel; every sum keeps the sequential
 * order (per-item terms are stored, then added in index order, and the
 * landmark contributions to the reduced system are added in landmark order),
 * so the results do not depend on the thread count. */
static int g_threads = 1;

/* Huber parameter of the robust norm (pixels); <= 0: squared norm. */
static double g_huber = 0.0;

void orc_set_huber(double delta) { g_huber = delta; }

/* rho(s) of the Huber norm for s = ||r||^2, and the IRLS weight w = rho'(s). */
static double huber_rho(double s) {
    if (!(g_huber > 0) || s <= g_huber * g_huber) return s;
    return 2.0 * g_huber * sqrt(s) - g_huber * g_huber;
}
static double huber_w(double s) {
    if (!(g_huber > 0) || s <= g_huber * g_huber) return 1.0;
    return g_huber / sqrt(s);
}

void orc_set_threads(int32_t n) { g_threads = n > 0 ? n : 1; }

int32_t orc_max_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_num_procs();
#else
    return 1;
#endif
}

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NUMERIC 5

/* ------------------------------------------------------------------------- */
/* rotations                                                                  */
/* ------------------------------------------------------------------------- */

/* Rotation matrix of axis-angle w (Rodrigues' formula), row-major. */
void orc_rotmat(const double w[3], double R[9]) {
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double a, b; /* R = I + a [w]x + b [w]x^2 */
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double kk = 0;
            for (int m = 0; m < 3; ++m) kk += K[i * 3 + m] * K[m * 3 + j];
            R[i * 3 + j] = (i == j ? 1.0 : 0.0) + a * K[i * 3 + j] + b * kk;
        }
}

static void quat_from_aa(const double w[3], double q[4]) {
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double s = th < 1e-8 ? 0.5 - th * th / 48.0 : sin(0.5 * th) / th;
    q[0] = cos(0.5 * th);
    q[1] = s * w[0];
    q[2] = s * w[1];
    q[3] = s * w[2];
}

static void aa_from_quat(const double qin[4], double w[3]) {
    double q[4] = {qin[0], qin[1], qin[2], qin[3]};
    if (q[0] < 0) for (int i = 0; i < 4; ++i) q[i] = -q[i];
    double vn = sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double f = vn < 1e-12 ? 2.0 / q[0] : 2.0 * atan2(vn, q[0]) / vn;
    w[0] = f * q[1];
    w[1] = f * q[2];
    w[2] = f * q[3];
}

/* out = Log(Exp(dw) Exp(w)) */
void orc_compose(const double dw[3], const double w[3], double out[3]) {
    double a[4], b[4], c[4];
    quat_from_aa(dw, a);
    quat_from_aa(w, b);
    c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    double n = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + c[3] * c[3]);
    for (int i = 0; i < 4; ++i) c[i] /= n;
    aa_from_quat(c, out);
}

/* ------------------------------------------------------------------------- */
/* camera model: residual and analytic Jacobians                               */
/* ------------------------------------------------------------------------- */

/* r = pi(cam, X) - z.  Jp: 2x9 row-major d r / d(dw, t, f, k1, k2);
 * Jl: 2x3 row-major d r / d X.  Either Jacobian pointer may be NULL. */
void orc_residual(const double cam[9], const double X[3], const double z[2],
                  double r[2], double Jp[18], double Jl[6]) {
    double R[9];
    orc_rotmat(cam, R);
    double Y[3], P[3];
    for (int i = 0; i < 3; ++i) {
        Y[i] = R[i * 3 + 0] * X[0] + R[i * 3 + 1] * X[1] + R[i * 3 + 2] * X[2];
        P[i] = Y[i] + cam[3 + i];
    }
    double f = cam[6], k1 = cam[7], k2 = cam[8];
    double p0 = -P[0] / P[2], p1 = -P[1] / P[2];
    double r2 = p0 * p0 + p1 * p1;
    double d = 1.0 + k1 * r2 + k2 * r2 * r2;
    r[0] = f * d * p0 - z[0];
    r[1] = f * d * p1 - z[1];
    if (!Jp && !Jl) return;

    /* d pixel / d p = f (d I + 2 (k1 + 2 k2 r2) p p^T) */
    double g = 2.0 * (k1 + 2.0 * k2 * r2);
    double Dp[4] = {f * (d + g * p0 * p0), f * g * p0 * p1,
                    f * g * p1 * p0, f * (d + g * p1 * p1)};
    /* d p / d P */
    double iz = 1.0 / P[2];
    double Pp[6] = {-iz, 0.0, P[0] * iz * iz,
                    0.0, -iz, P[1] * iz * iz};
    double A[6]; /* d pixel / d P, 2x3 */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            A[i * 3 + j] = Dp[i * 2 + 0] * Pp[0 * 3 + j] + Dp[i * 2 + 1] * Pp[1 * 3 + j];
    if (Jp) {
        /* dP/d(dw) = -[Y]x */
        double nYx[9] = {0, Y[2], -Y[1], -Y[2], 0, Y[0], Y[1], -Y[0], 0};
        for (int i = 0; i < 2; ++i) {
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int m = 0; m < 3; ++m) s += A[i * 3 + m] * nYx[m * 3 + j];
                Jp[i * 9 + j] = s;
                Jp[i * 9 + 3 + j] = A[i * 3 + j];
            }
        }
        double pp[2] = {p0, p1};
        for (int i = 0; i < 2; ++i) {
            Jp[i * 9 + 6] = d * pp[i];
            Jp[i * 9 + 7] = f * r2 * pp[i];
            Jp[i * 9 + 8] = f * r2 * r2 * pp[i];
        }
    }
    if (Jl) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int m = 0; m < 3; ++m) s += A[i * 3 + m] * R[m * 3 + j];
                Jl[i * 3 + j] = s;
            }
    }
}

/* Apply the update x <- x (+) dx: rotation by Exp(dw) from the left,
 * everything else additive. */
void orc_apply_update(int32_t n_cam, const double* cams, const double* dcams,
                      int32_t n_pt, const double* pts, const double* dpts,
                      double* cams_out, double* pts_out) {
    for (int32_t i = 0; i < n_cam; ++i) {
        double w[3];
        orc_compose(dcams + 9 * i, cams + 9 * i, w);
        for (int j = 0; j < 3; ++j) cams_out[9 * i + j] = w[j];
        for (int j = 3; j < 9; ++j) cams_out[9 * i + j] = cams[9 * i + j] + dcams[9 * i + j];
    }
    for (int64_t i = 0; i < 3 * (int64_t)n_pt; ++i) pts_out[i] = pts[i] + dpts[i];
}

/* E = sum ||r||^2 (Eq. ba_energy, no factor 1/2) */
double orc_cost(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                const double* obs_xy) {
    (void)n_cam;
    (void)n_pt;
    double* e = (double*)malloc(sizeof(double) * (n_obs + 1));
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t o = 0; o < n_obs; ++o) {
        double r[2];
        orc_residual(cams + 9 * obs_cam[o], pts + 3 * obs_pt[o], obs_xy + 2 * o, r, NULL, NULL);
        e[o] = huber_rho(r[0] * r[0] + r[1] * r[1]);
    }
    double E = 0;
    for (int64_t o = 0; o < n_obs; ++o) E += e[o];
    free(e);
    return E;
}

/* ------------------------------------------------------------------------- */
/* grouping observations by landmark (Sec. 5.1)                                */
/* ------------------------------------------------------------------------- */

static const int32_t* g_sort_pt;
static const int32_t* g_sort_cam;
static int cmp_obs(const void* a, const void* b) {
    int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
    if (g_sort_pt[i] != g_sort_pt[j]) return g_sort_pt[i] < g_sort_pt[j] ? -1 : 1;
    if (g_sort_cam[i] != g_sort_cam[j]) return g_sort_cam[i] < g_sort_cam[j] ? -1 : 1;
    return i < j ? -1 : (i > j);
}

/* perm[n_obs]: observation indices ordered by (landmark, camera).
 * pt_off[n_pt+1]: landmark j owns perm[pt_off[j] .. pt_off[j+1]).
 * cam_off[n_cam+1], cam_list[n_obs]: camera i owns the sorted-order positions
 * cam_list[cam_off[i] .. cam_off[i+1]) in increasing order.
 * Returns ORC_ERR_ARG on an index out of range, a landmark with fewer than
 * two observations, or a duplicate (landmark, camera) pair. */
int orc_sort_obs(int32_t n_cam, int32_t n_pt, int64_t n_obs, const int32_t* obs_cam,
                 const int32_t* obs_pt, int32_t* perm, int64_t* pt_off,
                 int64_t* cam_off, int32_t* cam_list) {
    for (int64_t o = 0; o < n_obs; ++o)
        if (obs_cam[o] < 0 || obs_cam[o] >= n_cam || obs_pt[o] < 0 || obs_pt[o] >= n_pt)
            return ORC_ERR_ARG;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (n_obs ? n_obs : 1));
    for (int64_t o = 0; o < n_obs; ++o) idx[o] = o;
    g_sort_pt = obs_pt;
    g_sort_cam = obs_cam;
    qsort(idx, (size_t)n_obs, sizeof(int64_t), cmp_obs);
    int rc = ORC_OK;
    for (int64_t j = 0; j <= n_pt; ++j) pt_off[j] = 0;
    for (int64_t o = 0; o < n_obs; ++o) {
        perm[o] = (int32_t)idx[o];
        pt_off[obs_pt[o] + 1]++;
        if (o > 0 && obs_pt[idx[o]] == obs_pt[idx[o - 1]] && obs_cam[idx[o]] == obs_cam[idx[o - 1]])
            rc = ORC_ERR_ARG;
    }
    for (int64_t j = 0; j < n_pt; ++j) {
        if (pt_off[j + 1] < 2) rc = ORC_ERR_ARG;
        pt_off[j + 1] += pt_off[j];
    }
    if (cam_off && cam_list) {
        for (int64_t i = 0; i <= n_cam; ++i) cam_off[i] = 0;
        for (int64_t o = 0; o < n_obs; ++o) cam_off[obs_cam[o] + 1]++;
        for (int64_t i = 0; i < n_cam; ++i) cam_off[i + 1] += cam_off[i];
        int64_t* fill = (int64_t*)calloc((size_t)n_cam + 1, sizeof(int64_t));
        for (int64_t s = 0; s < n_obs; ++s) { /* sorted positions, increasing */
            int32_t c = obs_cam[idx[s]];
            cam_list[cam_off[c] + fill[c]++] = (int32_t)s;
        }
        free(fill);
    }
    free(idx);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* small dense helpers                                                         */
/* ------------------------------------------------------------------------- */

/* In-place Cholesky of an n x n SPD matrix (lower factor, row-major).
 * Returns 0 on success, -1 if a pivot is not positive. */
static int chol(int n, double* A) {
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0)) return -1;
        double l = sqrt(s);
        A[j * n + j] = l;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / l;
        }
        for (int i = 0; i < j; ++i) A[i * n + j] = 0.0;
    }
    return 0;
}

/* Solve (L L^T) x = b in place (L from chol). */
static void chol_solve(int n, const double* L, double* x) {
    for (int i = 0; i < n; ++i) {
        double s = x[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------------- */
/* the problem at one linearisation point                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n_cam, n_pt;
    int64_t n_obs;
    const int32_t *obs_cam, *obs_pt;
    const double* obs_xy;
    int32_t* perm;       /* sorted order */
    int64_t* pt_off;
    /* per sorted observation */
    double* r;   /* 2 (rows scaled by sqrt(w) under the robust norm) */
    double* Jp;  /* 18 */
    double* Jl;  /* 6 */
    double* rho; /* rho(||r||^2) of the unscaled residual */
    double* Dp2; /* 9 n_cam */
    double* Dl2; /* 3 n_pt */
    /* block-sparse upper triangle of the RCS, 9x9 blocks */
    int64_t* row_ptr; /* n_cam + 1 */
    int32_t* col;     /* nblk */
    int64_t nblk;
    double* blk;      /* nblk * 81 */
    double* bt;       /* 9 n_cam: b~ = b_p - H_pl H_ll^-1 b_l */
    double lambda;
} orc_lin;

static int64_t find_block(const orc_lin* L, int32_t a, int32_t b) {
    int64_t lo = L->row_ptr[a], hi = L->row_ptr[a + 1] - 1;
    while (lo <= hi) {
        int64_t m = (lo + hi) / 2;
        if (L->col[m] == b) return m;
        if (L->col[m] < b) lo = m + 1; else hi = m - 1;
    }
    return -1;
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : (x > y);
}

static void lin_free(orc_lin* L) {
    free(L->perm); free(L->pt_off); free(L->r); free(L->Jp); free(L->Jl); free(L->rho);
    free(L->Dp2); free(L->Dl2); free(L->row_ptr); free(L->col); free(L->blk); free(L->bt);
    memset(L, 0, sizeof(*L));
}

/* Residuals, Jacobians, damping diagonals and the RCS sparsity pattern. */
static int lin_setup(orc_lin* L, int32_t n_cam, const double* cams, int32_t n_pt,
                     const double* pts, int64_t n_obs, const int32_t* obs_cam,
                     const int32_t* obs_pt, const double* obs_xy) {
    memset(L, 0, sizeof(*L));
    L->n_cam = n_cam; L->n_pt = n_pt; L->n_obs = n_obs;
    L->obs_cam = obs_cam; L->obs_pt = obs_pt; L->obs_xy = obs_xy;
    L->perm = (int32_t*)malloc(sizeof(int32_t) * (n_obs + 1));
    L->pt_off = (int64_t*)malloc(sizeof(int64_t) * (n_pt + 1));
    int rc = orc_sort_obs(n_cam, n_pt, n_obs, obs_cam, obs_pt, L->perm, L->pt_off, NULL, NULL);
    if (rc) return rc;
    L->r = (double*)malloc(sizeof(double) * 2 * (n_obs + 1));
    L->Jp = (double*)malloc(sizeof(double) * 18 * (n_obs + 1));
    L->Jl = (double*)malloc(sizeof(double) * 6 * (n_obs + 1));
    L->rho = (double*)malloc(sizeof(double) * (n_obs + 1));
    L->Dp2 = (double*)calloc(9 * (size_t)n_cam + 1, sizeof(double));
    L->Dl2 = (double*)calloc(3 * (size_t)n_pt + 1, sizeof(double));
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t s = 0; s < n_obs; ++s) {
        int32_t o = L->perm[s];
        orc_residual(cams + 9 * obs_cam[o], pts + 3 * obs_pt[o], obs_xy + 2 * o,
                     L->r + 2 * s, L->Jp + 18 * s, L->Jl + 6 * s);
        /* IRLS: the observation's rows scaled by sqrt(w) */
        const double sq = L->r[2 * s] * L->r[2 * s] + L->r[2 * s + 1] * L->r[2 * s + 1];
        L->rho[s] = huber_rho(sq);
        const double sw = sqrt(huber_w(sq));
        if (sw != 1.0) {
            for (int i = 0; i < 2; ++i) L->r[2 * s + i] *= sw;
            for (int i = 0; i < 18; ++i) L->Jp[18 * s + i] *= sw;
            for (int i = 0; i < 6; ++i) L->Jl[6 * s + i] *= sw;
        }
    }
    for (int64_t s = 0; s < n_obs; ++s) {
        int32_t o = L->perm[s];
        for (int c = 0; c < 9; ++c)
            L->Dp2[9 * obs_cam[o] + c] += L->Jp[18 * s + c] * L->Jp[18 * s + c] +
                                          L->Jp[18 * s + 9 + c] * L->Jp[18 * s + 9 + c];
        for (int c = 0; c < 3; ++c)
            L->Dl2[3 * obs_pt[o] + c] += L->Jl[6 * s + c] * L->Jl[6 * s + c] +
                                         L->Jl[6 * s + 3 + c] * L->Jl[6 * s + 3 + c];
    }
    for (int64_t i = 0; i < 9 * (int64_t)n_cam; ++i) L->Dp2[i] = clampd(L->Dp2[i], 1e-6, 1e32);
    for (int64_t i = 0; i < 3 * (int64_t)n_pt; ++i) L->Dl2[i] = clampd(L->Dl2[i], 1e-6, 1e32);

    /* pattern: (a, b), a <= b, for every pair of cameras sharing a landmark */
    int64_t npair = 0;
    for (int32_t j = 0; j < n_pt; ++j) {
        int64_t k = L->pt_off[j + 1] - L->pt_off[j];
        npair += k * (k + 1) / 2;
    }
    int64_t* keys = (int64_t*)malloc(sizeof(int64_t) * (npair + 1));
    int64_t q = 0;
    for (int32_t j = 0; j < n_pt; ++j)
        for (int64_t s = L->pt_off[j]; s < L->pt_off[j + 1]; ++s)
            for (int64_t t = s; t < L->pt_off[j + 1]; ++t) {
                int64_t a = obs_cam[L->perm[s]], b = obs_cam[L->perm[t]];
                keys[q++] = a * n_cam + b; /* sorted by cam within a landmark: a < b */
            }
    /* diagonal blocks for every camera, observed or not */
    int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (npair + n_cam + 1));
    memcpy(all, keys, sizeof(int64_t) * npair);
    for (int32_t i = 0; i < n_cam; ++i) all[npair + i] = (int64_t)i * n_cam + i;
    free(keys);
    int64_t tot = npair + n_cam;
    qsort(all, (size_t)tot, sizeof(int64_t), cmp_i64);
    int64_t u = 0;
    for (int64_t i = 0; i < tot; ++i)
        if (u == 0 || all[i] != all[u - 1]) all[u++] = all[i];
    L->nblk = u;
    L->row_ptr = (int64_t*)calloc((size_t)n_cam + 1, sizeof(int64_t));
    L->col = (int32_t*)malloc(sizeof(int32_t) * (u + 1));
    for (int64_t i = 0; i < u; ++i) {
        L->row_ptr[all[i] / n_cam + 1]++;
        L->col[i] = (int32_t)(all[i] % n_cam);
    }
    for (int32_t i = 0; i < n_cam; ++i) L->row_ptr[i + 1] += L->row_ptr[i];
    free(all);
    L->blk = (double*)malloc(sizeof(double) * 81 * (u + 1));
    L->bt = (double*)malloc(sizeof(double) * 9 * ((size_t)n_cam + 1));
    return ORC_OK;
}

/* Per-landmark damped Schur-complement pieces (Sec. 4.2 with the damped
 * H_ll + lambda D_l^2).  k = number of observations, slots in sorted order.
 *   Hll_d (3x3) = sum Jl^T Jl + lambda diag(Dl2)
 *   W_s   (9x3) = Jp_s^T Jl_s,  bl = sum Jl^T r,  bp_s = Jp_s^T r_s
 * S[s][t] (9x9) = [s==t] Jp_s^T Jp_s - W_s Hll_d^-1 W_t^T
 * bt_s (9)      = bp_s - W_s Hll_d^-1 bl
 * Returns -1 if Hll_d is not positive definite. */
static int landmark_sc(const orc_lin* L, int32_t j, double lambda, double* S /* (9k)^2 or NULL */,
                       double* bts /* 9k */, double* Hll_out /* 9 or NULL */,
                       double* cc_out /* reduced residual norm^2 or NULL */) {
    int64_t s0 = L->pt_off[j], k = L->pt_off[j + 1] - s0;
    double H[9] = {0}, bl[3] = {0};
    for (int64_t s = 0; s < k; ++s) {
        const double* Jl = L->Jl + 6 * (s0 + s);
        const double* r = L->r + 2 * (s0 + s);
        for (int a = 0; a < 3; ++a) {
            bl[a] += Jl[a] * r[0] + Jl[3 + a] * r[1];
            for (int b = 0; b < 3; ++b) H[a * 3 + b] += Jl[a] * Jl[b] + Jl[3 + a] * Jl[3 + b];
        }
    }
    for (int a = 0; a < 3; ++a) H[a * 3 + a] += lambda * L->Dl2[3 * j + a];
    if (Hll_out) memcpy(Hll_out, H, sizeof(H));
    double C[9];
    memcpy(C, H, sizeof(H));
    if (chol(3, C)) return -1;
    /* Y = Hll_d^-1 [W_1^T ... W_k^T | bl]  (3 x (9k+1)) */
    int64_t nc = 9 * k + 1;
    double* Y = (double*)malloc(sizeof(double) * 3 * nc);
    double* Wt = (double*)malloc(sizeof(double) * 3 * nc); /* [W^T | bl] */
    for (int64_t s = 0; s < k; ++s) {
        const double* Jp = L->Jp + 18 * (s0 + s);
        const double* Jl = L->Jl + 6 * (s0 + s);
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 9; ++c)
                Wt[a * nc + 9 * s + c] = Jl[a] * Jp[c] + Jl[3 + a] * Jp[9 + c];
    }
    for (int a = 0; a < 3; ++a) Wt[a * nc + 9 * k] = bl[a];
    for (int64_t c = 0; c < nc; ++c) {
        double x[3] = {Wt[0 * nc + c], Wt[1 * nc + c], Wt[2 * nc + c]};
        chol_solve(3, C, x);
        for (int a = 0; a < 3; ++a) Y[a * nc + c] = x[a];
    }
    int64_t n = 9 * k;
    if (S) {
        for (int64_t u = 0; u < n; ++u)
            for (int64_t v = 0; v < n; ++v) {
                double s = 0;
                for (int a = 0; a < 3; ++a) s += Wt[a * nc + u] * Y[a * nc + v];
                S[u * n + v] = -s;
            }
        for (int64_t s = 0; s < k; ++s) {
            const double* Jp = L->Jp + 18 * (s0 + s);
            for (int a = 0; a < 9; ++a)
                for (int b = 0; b < 9; ++b)
                    S[(9 * s + a) * n + 9 * s + b] += Jp[a] * Jp[b] + Jp[9 + a] * Jp[9 + b];
        }
    }
    for (int64_t s = 0; s < k; ++s) {
        const double* Jp = L->Jp + 18 * (s0 + s);
        const double* r = L->r + 2 * (s0 + s);
        for (int c = 0; c < 9; ++c) {
            double v = Jp[c] * r[0] + Jp[9 + c] * r[1];
            for (int a = 0; a < 3; ++a) v -= Wt[a * nc + 9 * s + c] * Y[a * nc + 9 * k];
            bts[9 * s + c] = v;
        }
    }
    if (cc_out) {
        double rr = 0;
        for (int64_t s = 0; s < k; ++s) {
            const double* r = L->r + 2 * (s0 + s);
            rr += r[0] * r[0] + r[1] * r[1];
        }
        for (int a = 0; a < 3; ++a) rr -= bl[a] * Y[a * nc + 9 * k];
        *cc_out = rr;
    }
    free(Y);
    free(Wt);
    return 0;
}

/* Assemble the damped RCS H~ (upper blocks incl. lambda D_p^2) and b~. */
static int lin_build_rcs(orc_lin* L, double lambda) {
    L->lambda = lambda;
    memset(L->blk, 0, sizeof(double) * 81 * L->nblk);
    memset(L->bt, 0, sizeof(double) * 9 * L->n_cam);
    int64_t kmax = 0;
    for (int32_t j = 0; j < L->n_pt; ++j) {
        int64_t k = L->pt_off[j + 1] - L->pt_off[j];
        if (k > kmax) kmax = k;
    }
    int rc = ORC_OK;
    /* each landmark's pieces are computed in parallel; they are added to the
     * blocks in landmark order (ordered region) */
#pragma omp parallel num_threads(g_threads)
    {
        double* S = (double*)malloc(sizeof(double) * 81 * kmax * kmax + 8);
        double* bts = (double*)malloc(sizeof(double) * 9 * kmax + 8);
#pragma omp for ordered schedule(dynamic, 1)
        for (int32_t j = 0; j < L->n_pt; ++j) {
            int64_t s0 = L->pt_off[j], k = L->pt_off[j + 1] - s0, n = 9 * k;
            int bad = landmark_sc(L, j, lambda, S, bts, NULL, NULL);
#pragma omp ordered
            {
                if (bad) rc = ORC_ERR_NUMERIC;
                for (int64_t s = 0; s < k && !bad; ++s) {
                    int32_t a = L->obs_cam[L->perm[s0 + s]];
                    for (int c = 0; c < 9; ++c) L->bt[9 * a + c] += bts[9 * s + c];
                    for (int64_t t = s; t < k; ++t) {
                        int32_t b = L->obs_cam[L->perm[s0 + t]];
                        int64_t bi = find_block(L, a, b);
                        double* B = L->blk + 81 * bi;
                        for (int u = 0; u < 9; ++u)
                            for (int v = 0; v < 9; ++v) B[u * 9 + v] += S[(9 * s + u) * n + 9 * t + v];
                    }
                }
            }
        }
        free(S);
        free(bts);
    }
    for (int32_t i = 0; i < L->n_cam; ++i) {
        double* B = L->blk + 81 * find_block(L, i, i);
        for (int u = 0; u < 9; ++u) B[u * 9 + u] += lambda * L->Dp2[9 * i + u];
    }
    return rc;
}

/* y = H~ x from the symmetric upper-block storage */
static void rcs_matvec(const orc_lin* L, const double* x, double* y) {
    memset(y, 0, sizeof(double) * 9 * L->n_cam);
    for (int32_t a = 0; a < L->n_cam; ++a)
        for (int64_t bi = L->row_ptr[a]; bi < L->row_ptr[a + 1]; ++bi) {
            int32_t b = L->col[bi];
            const double* B = L->blk + 81 * bi;
            for (int u = 0; u < 9; ++u)
                for (int v = 0; v < 9; ++v) {
                    y[9 * a + u] += B[u * 9 + v] * x[9 * b + v];
                    if (a != b) y[9 * b + v] += B[u * 9 + v] * x[9 * a + u];
                }
        }
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Products y = H x of the operator a PCG run iterates on. */
typedef void (*orc_matvec_fn)(const void* ctx, const double* x, double* y);

/* Block-Jacobi PCG on H dx = g (Sec. 5.4 / 6.1) for n_blk blocks of 9 unknowns.
 * Mblk holds the n_blk diagonal 9x9 blocks of H (row-major), mv applies H.
 * Stop rules (reading of the "forcing sequence" of Sec. 6.1): the truncated-Newton
 * test of Nash and Sofer i (Q_i - Q_{i-1}) / Q_i < eta with Q(x) = 1/2 x^T H x - g^T x
 * evaluated as -1/2 x^T (g + r) and Q_0 = Q(0) = 0; ||r_i|| <= 1e-10 ||g||; i = max_it.
 * x starts at 0.  Qlog (max_it + 1 entries, or NULL) receives Q_0 .. Q_i.
 * Returns the number of iterations; *status = 0 ok, 1 breakdown. */
static int pcg_block_jacobi(int32_t n_blk, orc_matvec_fn mv, const void* ctx,
                            const double* Mblk, const double* g, double* x, int max_it,
                            double eta, int* status, double* Qlog) {
    int64_t n = 9 * (int64_t)n_blk;
    double* Minv = (double*)malloc(sizeof(double) * 81 * (n_blk > 0 ? n_blk : 1));
    *status = 0;
    for (int32_t i = 0; i < n_blk; ++i) {
        memcpy(Minv + 81 * i, Mblk + 81 * i, sizeof(double) * 81);
        if (chol(9, Minv + 81 * i)) *status = 1;
    }
    double *r = (double*)malloc(sizeof(double) * (n + 1)), *z = (double*)malloc(sizeof(double) * (n + 1));
    double *p = (double*)malloc(sizeof(double) * (n + 1)), *q = (double*)malloc(sizeof(double) * (n + 1));
    double* tmp = (double*)malloc(sizeof(double) * (n + 1));
    memset(x, 0, sizeof(double) * n);
    memcpy(r, g, sizeof(double) * n);
    double gnorm = sqrt(dot(n, g, g));
    int it = 0;
    if (Qlog) Qlog[0] = 0.0;
    if (*status || gnorm == 0) goto done;
    for (int32_t i = 0; i < n_blk; ++i) {
        memcpy(z + 9 * i, r + 9 * i, sizeof(double) * 9);
        chol_solve(9, Minv + 81 * i, z + 9 * i);
    }
    memcpy(p, z, sizeof(double) * n);
    double rho = dot(n, r, z), Q0 = 0.0;
    for (it = 1; it <= max_it; ++it) {
        mv(ctx, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0)) { *status = 1; it -= 1; break; }
        double alpha = rho / pq;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        for (int64_t i = 0; i < n; ++i) tmp[i] = g[i] + r[i];
        double Q1 = -0.5 * dot(n, x, tmp);
        if (Qlog) Qlog[it] = Q1;
        if (sqrt(dot(n, r, r)) <= 1e-10 * gnorm) break;
        if (it * (Q1 - Q0) / Q1 < eta) break;
        Q0 = Q1;
        if (it == max_it) break;
        for (int32_t i = 0; i < n_blk; ++i) {
            memcpy(z + 9 * i, r + 9 * i, sizeof(double) * 9);
            chol_solve(9, Minv + 81 * i, z + 9 * i);
        }
        double rho1 = dot(n, r, z);
        double beta = rho1 / rho;
        rho = rho1;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it > max_it) it = max_it;
done:
    free(Minv); free(r); free(z); free(p); free(q); free(tmp);
    return it;
}

static void rcs_matvec_cb(const void* ctx, const double* x, double* y) {
    rcs_matvec((const orc_lin*)ctx, x, y);
}

/* Block-Jacobi PCG on the damped RCS H~ dx = g with g = -b~, preconditioned by
 * the diagonal blocks of H~ (Sec. 5.4). */
static int rcs_pcg(const orc_lin* L, const double* g, double* x, int max_it, double eta,
                   int* status) {
    double* Mblk = (double*)malloc(sizeof(double) * 81 * (L->n_cam > 0 ? L->n_cam : 1));
    for (int32_t i = 0; i < L->n_cam; ++i)
        memcpy(Mblk + 81 * i, L->blk + 81 * find_block(L, i, i), sizeof(double) * 81);
    int it = pcg_block_jacobi(L->n_cam, rcs_matvec_cb, L, Mblk, g, x, max_it, eta, status, NULL);
    free(Mblk);
    return it;
}

typedef struct {
    int64_t n;
    const double* H;
} dense_op;

static void dense_matvec_cb(const void* ctx, const double* x, double* y) {
    const dense_op* d = (const dense_op*)ctx;
    for (int64_t i = 0; i < d->n; ++i) {
        double s = 0;
        for (int64_t j = 0; j < d->n; ++j) s += d->H[i * d->n + j] * x[j];
        y[i] = s;
    }
}

/* The same PCG on a dense SPD matrix H (9 n_blk square, row-major), block-Jacobi
 * preconditioned by its 9x9 diagonal blocks.  Exposed so that the stop rule can be
 * checked on systems whose CG iterates are known independently.  Returns the
 * iteration count; *status as above; Qlog as above (may be NULL). */
int orc_pcg_dense(int32_t n_blk, const double* H, const double* g, int32_t max_it, double eta,
                  double* x, double* Qlog, int32_t* status) {
    int64_t n = 9 * (int64_t)n_blk;
    double* Mblk = (double*)malloc(sizeof(double) * 81 * (n_blk > 0 ? n_blk : 1));
    for (int32_t b = 0; b < n_blk; ++b)
        for (int u = 0; u < 9; ++u)
            for (int v = 0; v < 9; ++v) Mblk[81 * b + 9 * u + v] = H[(9 * b + u) * n + 9 * b + v];
    dense_op d = {n, H};
    int st = 0;
    int it = pcg_block_jacobi(n_blk, dense_matvec_cb, &d, Mblk, g, x, max_it, eta, &st, Qlog);
    *status = st;
    free(Mblk);
    return it;
}

/* Dense H~ (n x n, both triangles) from the block storage. */
static void rcs_dense(const orc_lin* L, double* D) {
    int64_t n = 9 * (int64_t)L->n_cam;
    memset(D, 0, sizeof(double) * n * n);
    for (int32_t a = 0; a < L->n_cam; ++a)
        for (int64_t bi = L->row_ptr[a]; bi < L->row_ptr[a + 1]; ++bi) {
            int32_t b = L->col[bi];
            const double* B = L->blk + 81 * bi;
            for (int u = 0; u < 9; ++u)
                for (int v = 0; v < 9; ++v) {
                    D[(9 * a + u) * n + 9 * b + v] = B[u * 9 + v];
                    D[(9 * b + v) * n + 9 * a + u] = B[u * 9 + v];
                }
        }
}

/* Landmark back substitution (Eq. backsub_sc, damped):
 * dl_j = -(H_ll + lambda D_l^2)^-1 (b_l + H_lp dp) */
static int lin_backsub(const orc_lin* L, const double* dp, double* dl) {
    int rc = ORC_OK;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int32_t j = 0; j < L->n_pt; ++j) {
        int64_t s0 = L->pt_off[j], k = L->pt_off[j + 1] - s0;
        double H[9] = {0}, v[3] = {0};
        for (int64_t s = 0; s < k; ++s) {
            const double* Jl = L->Jl + 6 * (s0 + s);
            const double* Jp = L->Jp + 18 * (s0 + s);
            const double* r = L->r + 2 * (s0 + s);
            const double* d = dp + 9 * L->obs_cam[L->perm[s0 + s]];
            double e[2] = {r[0], r[1]}; /* r + Jp dp */
            for (int c = 0; c < 9; ++c) { e[0] += Jp[c] * d[c]; e[1] += Jp[9 + c] * d[c]; }
            for (int a = 0; a < 3; ++a) {
                v[a] += Jl[a] * e[0] + Jl[3 + a] * e[1];
                for (int b = 0; b < 3; ++b) H[a * 3 + b] += Jl[a] * Jl[b] + Jl[3 + a] * Jl[3 + b];
            }
        }
        for (int a = 0; a < 3; ++a) H[a * 3 + a] += L->lambda * L->Dl2[3 * j + a];
        if (chol(3, H)) {
            rc = ORC_ERR_NUMERIC; /* any thread: the same status */
            continue;
        }
        chol_solve(3, H, v);
        for (int a = 0; a < 3; ++a) dl[3 * j + a] = -v[a];
    }
    return rc;
}

/* Model cost L(dx) = ||r + J dx||^2 (undamped). */
static double lin_model_cost(const orc_lin* L, const double* dp, const double* dl) {
    double* t = (double*)malloc(sizeof(double) * (L->n_obs + 1));
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t s = 0; s < L->n_obs; ++s) {
        double m = 0;
        int32_t o = L->perm[s];
        const double* Jp = L->Jp + 18 * s;
        const double* Jl = L->Jl + 6 * s;
        const double* d = dp + 9 * L->obs_cam[o];
        const double* e = dl + 3 * L->obs_pt[o];
        for (int i = 0; i < 2; ++i) {
            double v = L->r[2 * s + i];
            for (int c = 0; c < 9; ++c) v += Jp[9 * i + c] * d[c];
            for (int c = 0; c < 3; ++c) v += Jl[3 * i + c] * e[c];
            m += v * v;
        }
        /* rho(s) - w ||r||^2 + w ||r + J dx||^2 (the rows are the scaled ones) */
        t[s] = L->rho[s] - (L->r[2 * s] * L->r[2 * s] + L->r[2 * s + 1] * L->r[2 * s + 1]) + m;
    }
    double m = 0;
    for (int64_t s = 0; s < L->n_obs; ++s) m += t[s];
    free(t);
    return m;
}

/* ------------------------------------------------------------------------- */
/* exported building blocks for the tests                                      */
/* ------------------------------------------------------------------------- */

/* Damping diagonals D_p^2 (9 n_cam) and D_l^2 (3 n_pt). */
int orc_damping_diag(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                     int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                     const double* obs_xy, double* Dp2, double* Dl2) {
    orc_lin L;
    int rc = lin_setup(&L, n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy);
    if (!rc) {
        memcpy(Dp2, L.Dp2, sizeof(double) * 9 * n_cam);
        memcpy(Dl2, L.Dl2, sizeof(double) * 3 * n_pt);
    }
    lin_free(&L);
    return rc;
}

/* Dense damped RCS H~ (N_p x N_p with N_p = 9 n_cam) and b~ (N_p). */
int orc_rcs_dense(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                  int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                  const double* obs_xy, double lambda, double* H, double* bt) {
    orc_lin L;
    int rc = lin_setup(&L, n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy);
    if (!rc) rc = lin_build_rcs(&L, lambda);
    if (!rc) {
        if (H) rcs_dense(&L, H);
        memcpy(bt, L.bt, sizeof(double) * 9 * n_cam);
    }
    lin_free(&L);
    return rc;
}

/* Per-camera diagonal blocks of H~ (n_cam x 81) and b~, block-sparse path. */
int orc_rcs_diag(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                 int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                 const double* obs_xy, double lambda, double* Mdiag, double* bt) {
    orc_lin L;
    int rc = lin_setup(&L, n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy);
    if (!rc) rc = lin_build_rcs(&L, lambda);
    if (!rc) {
        for (int32_t i = 0; i < n_cam; ++i)
            memcpy(Mdiag + 81 * i, L.blk + 81 * find_block(&L, i, i), sizeof(double) * 81);
        memcpy(bt, L.bt, sizeof(double) * 9 * n_cam);
    }
    lin_free(&L);
    return rc;
}

/* Per-landmark damped SC pieces for landmark j (slots in camera order):
 * S (9k x 9k), bts (9k), Hll_d (3x3), reduced residual norm^2.  *k_out = k. */
int orc_landmark_sc(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                    int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                    const double* obs_xy, double lambda, int32_t j, int32_t k_cap,
                    double* S, double* bts, double* Hll, double* cc, int32_t* k_out) {
    orc_lin L;
    int rc = lin_setup(&L, n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy);
    if (!rc && (j < 0 || j >= n_pt)) rc = ORC_ERR_ARG;
    if (!rc) {
        int64_t k = L.pt_off[j + 1] - L.pt_off[j];
        *k_out = (int32_t)k;
        if (k > k_cap) rc = ORC_ERR_ARG;
        else if (landmark_sc(&L, j, lambda, S, bts, Hll, cc)) rc = ORC_ERR_NUMERIC;
    }
    lin_free(&L);
    return rc;
}

/* y = H~ v with the damped Schur complement assembled block-sparse. */
int orc_rcs_matvec(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                   int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                   const double* obs_xy, double lambda, int32_t nv, const double* v, double* y) {
    orc_lin L;
    int rc = lin_setup(&L, n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy);
    if (!rc) rc = lin_build_rcs(&L, lambda);
    for (int32_t m = 0; !rc && m < nv; ++m)
        rcs_matvec(&L, v + 9 * (int64_t)n_cam * m, y + 9 * (int64_t)n_cam * m);
    lin_free(&L);
    return rc;
}

/* Landmark back substitution (Eq. backsub_sc, damped) for a given pose
 * step dp, and the model cost L(dx) = ||r + J dx||^2 of the full step. */
int orc_backsub_given(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                      int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                      const double* obs_xy, double lambda, const double* dp, double* dl,
                      double* model_cost) {
    orc_lin L;
    int rc = lin_setup(&L, n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy);
    L.lambda = lambda;
    if (!rc) rc = lin_backsub(&L, dp, dl);
    if (!rc) *model_cost = lin_model_cost(&L, dp, dl);
    lin_free(&L);
    return rc;
}

typedef struct {
    double lambda0;   /* 1e-4 */
    int32_t max_iters; /* 50 */
    double func_tol;  /* 1e-6 */
    int32_t max_cg;   /* 500 */
    double cg_eta;    /* 0.1 */
    int32_t dense;    /* 1: dense Cholesky RCS solve, 0: block-Jacobi PCG */
    double target_cost; /* > 0: also stop at the first accepted cost <= target (timing hook) */
} orc_options;

/* One damped linear step at the given state: dp (9 n_cam), dl (3 n_pt),
 * model cost L(dx) and the current cost E; returns CG iterations in *cg. */
int orc_linear_step(int32_t n_cam, const double* cams, int32_t n_pt, const double* pts,
                    int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                    const double* obs_xy, double lambda, const orc_options* opt,
                    double* dp, double* dl, double* model_cost, double* cost,
                    int32_t* cg) {
    orc_lin L;
    int rc = lin_setup(&L, n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy);
    if (!rc) rc = lin_build_rcs(&L, lambda);
    int64_t n = 9 * (int64_t)n_cam;
    if (!rc) {
        double* g = (double*)malloc(sizeof(double) * n);
        for (int64_t i = 0; i < n; ++i) g[i] = -L.bt[i];
        *cg = 0;
        if (opt->dense) {
            double* D = (double*)malloc(sizeof(double) * n * n);
            rcs_dense(&L, D);
            if (chol((int)n, D)) rc = ORC_ERR_NUMERIC;
            else { memcpy(dp, g, sizeof(double) * n); chol_solve((int)n, D, dp); }
            free(D);
        } else {
            int st = 0;
            *cg = rcs_pcg(&L, g, dp, opt->max_cg, opt->cg_eta, &st);
        }
        free(g);
    }
    if (!rc) rc = lin_backsub(&L, dp, dl);
    if (!rc) {
        *model_cost = lin_model_cost(&L, dp, dl);
        double E = 0;
        for (int64_t s = 0; s < n_obs; ++s) E += L.rho[s];
        *cost = E;
    }
    lin_free(&L);
    return rc;
}

typedef struct {
    double cost;        /* E at the start of the iteration */
    double new_cost;    /* E at the candidate */
    double model_cost;  /* L(dx) */
    double lambda;      /* damping used for this iteration */
    double rho;
    int32_t cg_iters;
    int32_t accepted;
} orc_iter;

/* The decision that ends one LM iteration (Sec. 6.1: the step is judged by the
 * ratio of actual and model cost reduction; the damping update follows Nielsen's
 * rule, the reading of "in line with Ceres").
 *   rho = (E - En) / (E - model); accept iff En and rho are finite, E - model > 0
 *   and rho > 1e-3.
 *   accept: lambda <- lambda * max(1/3, 1 - (2 rho - 1)^3), nu <- 2, lambda >= 1e-16;
 *           stop when |E - En| / E < func_tol, or when target_cost > 0 and En <= target_cost.
 *   reject: lambda <- lambda * nu, nu <- 2 nu; stop when lambda >= 1e32.
 * Returns 1 if the step is accepted; *stop is set to 1 when the loop ends here. */
int orc_lm_decide(double E, double En, double model, double func_tol, double target_cost,
                  double* lambda, double* nu, int32_t* stop, double* rho_out) {
    double rho = (E - En) / (E - model);
    int acc = isfinite(En) && isfinite(rho) && (E - model) > 0 && rho > 1e-3;
    *stop = 0;
    if (rho_out) *rho_out = rho;
    if (acc) {
        double t = 2.0 * rho - 1.0;
        double f = 1.0 - t * t * t;
        *lambda *= f > 1.0 / 3.0 ? f : 1.0 / 3.0;
        *nu = 2.0;
        if (*lambda < 1e-16) *lambda = 1e-16;
        if (fabs(E - En) / E < func_tol) *stop = 1;
        if (target_cost > 0 && En <= target_cost) *stop = 1;
    } else {
        *lambda *= *nu;
        *nu *= 2.0;
        if (*lambda >= 1e32) *stop = 1;
    }
    return acc;
}

/* Levenberg-Marquardt (Sec. 6.1).  cams/pts are updated in place.
 * log has room for opt->max_iters entries; *n_log receives the count. */
int orc_lm(int32_t n_cam, double* cams, int32_t n_pt, double* pts, int64_t n_obs,
           const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_xy,
           const orc_options* opt, orc_iter* log, int32_t* n_log) {
    double lambda = opt->lambda0, nu = 2.0;
    int64_t np = 9 * (int64_t)n_cam, nl = 3 * (int64_t)n_pt;
    double* dp = (double*)malloc(sizeof(double) * (np + 1));
    double* dl = (double*)malloc(sizeof(double) * (nl + 1));
    double* cn = (double*)malloc(sizeof(double) * (np + 1));
    double* pn = (double*)malloc(sizeof(double) * (nl + 1));
    int rc = ORC_OK;
    *n_log = 0;
    for (int32_t it = 0; it < opt->max_iters; ++it) {
        double model, E;
        int32_t cg = 0;
        rc = orc_linear_step(n_cam, cams, n_pt, pts, n_obs, obs_cam, obs_pt, obs_xy, lambda,
                             opt, dp, dl, &model, &E, &cg);
        if (rc) break;
        orc_apply_update(n_cam, cams, dp, n_pt, pts, dl, cn, pn);
        double En = orc_cost(n_cam, cn, n_pt, pn, n_obs, obs_cam, obs_pt, obs_xy);
        double lam_it = lambda, rho = 0;
        int32_t stop = 0;
        int acc = orc_lm_decide(E, En, model, opt->func_tol, opt->target_cost, &lambda, &nu,
                                &stop, &rho);
        orc_iter* lg = log + (*n_log)++;
        lg->cost = E; lg->new_cost = En; lg->model_cost = model; lg->lambda = lam_it;
        lg->rho = rho; lg->cg_iters = cg; lg->accepted = acc;
        if (acc) {
            memcpy(cams, cn, sizeof(double) * np);
            memcpy(pts, pn, sizeof(double) * nl);
        }
        if (stop) break;
    }
    free(dp); free(dl); free(cn); free(pn);
    return rc;
}
