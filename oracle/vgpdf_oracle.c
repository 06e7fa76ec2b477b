/*
 * vgpdf_oracle.c -- plain, slow, FP64 CPU oracle for batched local-GP distance fields.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header, table or
 * constant with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes, in the paper's order (Wu, Le Gentil, Vidal-Calleja, "VDB-GPDF",
 * arXiv 2407.09649):
 *   - voxelisation into 8^3-voxel leaves, voxel centres as training points (Sec. IV-A);
 *   - one GP per leaf / per query neighbourhood, SE kernel k = exp(-r^2 / (2 l^2))
 *     (Sec. III-A), A = K + sigma^2 I factorised by a textbook Cholesky, alpha = A^-1 1
 *     (Eq. 1);
 *   - latent mean o = k^T alpha (Eq. 1), latent variance u = 1 - k^T A^-1 k (Eq. 2 with
 *     the sign read as the standard GP posterior), gradient of o (Eq. 5);
 *   - reverting d = sqrt(-2 l^2 log o) (Eq. 3), distance variance v = Lambda^2 u with
 *     Lambda = -l / (o sqrt(-2 log o)) = -l^2 / (o d) (Eq. 4), chain-rule gradient
 *     grad d = -l^2 grad o / (o d);
 *   - closest-node selection of the L-GPDF GP for each testing voxel (Sec. IV-B);
 *   - probabilistic fusion, inverse-variance (Eqs. 7-8) or TSDF-style weights (Eq. 9);
 *   - G-GPDF queries against the GP of the query's 27-leaf neighbourhood (Sec. IV-D,
 *     with the neighbourhood search done on the leaf lattice instead of a kd-tree);
 *   - the backward pass of the distance w.r.t. query and surface points, derived from
 *     Eq. 1 by differentiating alpha = A^-1 1;
 *   - zero crossings and marching cubes over the fused grid, restricted to the leaves the
 *     latest fusion touched (Sec. IV-D): the G-GPDF training points and the mesh;
 *   - surface properties (Eq. 6): each voxel's property is the mean of its points'; per leaf
 *     a GP with the same kernel and noise sigma_prop gives c = k^T (K + sigma_prop^2 I)^-1 y
 *     and w = 1 - k^T (K + sigma_prop^2 I)^-1 k at the testing voxels; they are fused with the
 *     rules of Eqs. 8-9 using w, where the distance is fused; crossings and mesh vertices
 *     carry the fused properties interpolated with the crossing's t.
 *
 * The paper leaves the following open; this file takes these readings:
 *   - voxel index ijk = floor(p / vs + 1/2) in IEEE FP64 (p widened from float32);
 *     |ijk| < 2^20 - 64, else the point is dropped / the query is invalid;
 *   - voxel bit inside a leaf = x + 8 y + 64 z of the in-leaf offset; training points
 *     of a leaf in ascending bit order; when a leaf holds n > cap occupied voxels it
 *     keeps indices floor(k n / cap), k = 0..cap-1;
 *   - the capped occupancy of Eq. 3-4: o >= 1 gives d = 0 with zero gradient;
 *     o <= 0 or log o below -d_max^2 / (2 l^2) gives d = d_max, status 2; Lambda uses
 *     max(d, d_var_floor) and o = 1 when o >= 1;
 *   - closest L-GPDF node: the voxel's own leaf if it holds a GP, else the neighbour leaf
 *     with the smallest squared centre distance in half-voxel integer units, ties to the
 *     first in (dz, dy, dx) order from -1 to 1;
 *   - G-GPDF instance of a query leaf M: the points of the 27 leaves around M; if those
 *     are empty, the 27 leaves around the nearest occupied leaf F within Chebyshev radius
 *     max_leaf_search (nearest by integer leaf distance, ties to the smaller key); none ->
 *     status 1.  When an instance has more than max_pts_group points it keeps those
 *     nearest to the centre leaf's centre (FP64 squared distance, ties to the lower
 *     point index); instance points are kept in ascending point index.
 *
 * Parity status: every exported function is pinned by the CPU tests against closed forms,
 * brute force, exact rational arithmetic or invariants.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off -fopenmp (no FMA contraction, so the
 * voxel-key and selection arithmetic is the plain IEEE sequence written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double voxel_size;      /* metres per voxel edge */
    double lengthscale;     /* SE kernel length scale l (m) */
    double sigma_occ;       /* latent occupancy noise std; sigma^2 is added to diag(K) */
    double d_max;           /* distance cap (m) -> log-occupancy floor */
    double d_var_floor;     /* lower bound on d inside Lambda (m) */
    int32_t max_pts_leaf;   /* per-leaf training cap (L-GPDF) */
    int32_t max_pts_group;  /* per-neighbourhood cap (G-GPDF) */
    int32_t max_leaf_search;/* Chebyshev leaf radius of the fallback search */
    int32_t fusion;         /* 0: inverse variance (Eqs. 7-8); 1: TSDF weights (Eq. 9) */
    double sigma_prop;      /* noise std of the surface-property GP (Eq. 6) */
    int32_t n_props;        /* property channels per point, 0..4 */
    int32_t pad_;
} or_params;

#define MAX_PROPS 4

enum { ST_OK = 0, ST_NO_SUPPORT = 1, ST_CLAMPED = 2, ST_BAD_INPUT = 3, ST_FACTOR_FAIL = 4 };

#define KEY_BIAS (1LL << 20)
#define IJK_LIMIT 1048512.0 /* 2^20 - 64 */

/* ------------------------------------------------------------------------------------ */
/* indexing                                                                             */
/* ------------------------------------------------------------------------------------ */
static int64_t floor_div8(int64_t v) { return v >= 0 ? v / 8 : -((-v + 7) / 8); }

static uint64_t pack_key(int64_t x, int64_t y, int64_t z) {
    return ((uint64_t)(x + KEY_BIAS) << 42) | ((uint64_t)(y + KEY_BIAS) << 21) |
           (uint64_t)(z + KEY_BIAS);
}

static void unpack_key(uint64_t k, int64_t out[3]) {
    out[0] = (int64_t)((k >> 42) & 0x1FFFFF) - KEY_BIAS;
    out[1] = (int64_t)((k >> 21) & 0x1FFFFF) - KEY_BIAS;
    out[2] = (int64_t)(k & 0x1FFFFF) - KEY_BIAS;
}

/* voxel index of one point (Sec. IV-A: points are grouped by the voxel they fall in). */
static int voxel_ijk(const double p[3], double vs, int64_t ijk[3]) {
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(p[a])) return 0;
        double t = p[a] / vs;
        double u = t + 0.5;
        double f = floor(u);
        if (!(f > -IJK_LIMIT && f < IJK_LIMIT)) return 0;
        ijk[a] = (int64_t)f;
    }
    return 1;
}

static void leaf_of(const int64_t ijk[3], int64_t leaf[3], int32_t* bit) {
    for (int a = 0; a < 3; ++a) leaf[a] = floor_div8(ijk[a]);
    *bit = (int32_t)((ijk[0] - 8 * leaf[0]) + 8 * (ijk[1] - 8 * leaf[1]) + 64 * (ijk[2] - 8 * leaf[2]));
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

static int64_t find_key(const uint64_t* keys, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < n && keys[lo] == k) ? lo : -1;
}

void or_index_points(const or_params* P, const float* pts, int64_t n, int64_t* ijk_out,
                     uint64_t* vkey, uint64_t* lkey, int32_t* bit_out, uint8_t* ok) {
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {(double)pts[3 * i], (double)pts[3 * i + 1], (double)pts[3 * i + 2]};
        int64_t ijk[3] = {0, 0, 0}, leaf[3] = {0, 0, 0};
        int32_t bit = 0;
        int good = voxel_ijk(p, P->voxel_size, ijk);
        if (good) leaf_of(ijk, leaf, &bit);
        if (ijk_out) for (int a = 0; a < 3; ++a) ijk_out[3 * i + a] = good ? ijk[a] : 0;
        if (vkey) vkey[i] = good ? pack_key(ijk[0], ijk[1], ijk[2]) : 0;
        if (lkey) lkey[i] = good ? pack_key(leaf[0], leaf[1], leaf[2]) : 0;
        if (bit_out) bit_out[i] = good ? bit : -1;
        if (ok) ok[i] = (uint8_t)good;
    }
}

/* ------------------------------------------------------------------------------------ */
/* dense GP algebra on one instance (Eqs. 1, 2, 5), packed lower triangle, row major     */
/* ------------------------------------------------------------------------------------ */
#define PK(i, j) ((int64_t)(i) * ((i) + 1) / 2 + (j))

/* Cholesky-Banachiewicz, row by row: A = L L^T, L overwrites the lower triangle. */
static int cholesky_packed(double* A, int N) {
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[PK(i, j)];
            for (int k = 0; k < j; ++k) s -= A[PK(i, k)] * A[PK(j, k)];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                A[PK(i, i)] = sqrt(s);
            } else {
                A[PK(i, j)] = s / A[PK(j, j)];
            }
        }
    }
    return 1;
}

/* L z = b (forward substitution) */
static void forward_subst(const double* L, int N, const double* b, double* z) {
    for (int i = 0; i < N; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[PK(i, k)] * z[k];
        z[i] = s / L[PK(i, i)];
    }
}

/* L^T x = z (back substitution) */
static void back_subst(const double* L, int N, const double* z, double* x) {
    for (int i = N - 1; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < N; ++k) s -= L[PK(k, i)] * x[k];
        x[i] = s / L[PK(i, i)];
    }
}

static double se_kernel(const double* a, const double* b, double l) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    return exp(-r2 / (2.0 * l * l));
}

/* Train one GP: L = chol(K + sigma^2 I), alpha = (K + sigma^2 I)^-1 1 (Eq. 1). */
int or_gp_fit(const double* X, int N, const or_params* P, double* L, double* alpha) {
    double s2 = P->sigma_occ * P->sigma_occ;
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < i; ++j) L[PK(i, j)] = se_kernel(X + 3 * i, X + 3 * j, P->lengthscale);
        L[PK(i, i)] = 1.0 + s2;
    }
    if (!cholesky_packed(L, N)) return 0;
    double* ones = (double*)malloc(sizeof(double) * (N > 0 ? N : 1));
    double* z = (double*)malloc(sizeof(double) * (N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) ones[i] = 1.0;
    forward_subst(L, N, ones, z);
    back_subst(L, N, z, alpha);
    free(ones);
    free(z);
    return 1;
}

typedef struct {
    double o, go[3], u, d, gd[3], v;
    int status;
} or_eval;

/* Reverting function (Eq. 3), its variance (Eq. 4) and the chain-rule gradient. */
static void revert(const or_params* P, or_eval* r) {
    double l = P->lengthscale, l2 = l * l;
    double log_floor = -(P->d_max * P->d_max) / (2.0 * l2);
    if (!(r->o > 0.0)) {
        r->status = ST_CLAMPED; r->d = P->d_max; r->gd[0] = r->gd[1] = r->gd[2] = 0.0;
        r->v = INFINITY;
        return;
    }
    double lo = log(r->o);
    if (lo < log_floor) {
        r->status = ST_CLAMPED; r->d = P->d_max; r->gd[0] = r->gd[1] = r->gd[2] = 0.0;
        r->v = INFINITY;
        return;
    }
    r->status = ST_OK;
    if (lo >= 0.0) {
        double lam = -l2 / (1.0 * P->d_var_floor);
        r->d = 0.0; r->gd[0] = r->gd[1] = r->gd[2] = 0.0;
        r->v = lam * lam * r->u;
        return;
    }
    r->d = sqrt(-2.0 * l2 * lo);
    for (int a = 0; a < 3; ++a) r->gd[a] = -l2 * r->go[a] / (r->o * r->d);
    double dv = r->d > P->d_var_floor ? r->d : P->d_var_floor;
    double lam = -l2 / (r->o * dv);
    r->v = lam * lam * r->u;
}

/* Latent mean (Eq. 1), its gradient (Eq. 5), latent variance (Eq. 2), then reverting. */
static void gp_eval(const double* X, int N, const double* L, const double* alpha,
                    const double xs[3], const or_params* P, int want_var, double* kbuf,
                    double* vbuf, or_eval* r) {
    double l = P->lengthscale;
    double o = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < N; ++j) {
        double k = se_kernel(xs, X + 3 * j, l);
        if (kbuf) kbuf[j] = k;
        o += alpha[j] * k;
        for (int a = 0; a < 3; ++a) g[a] += alpha[j] * k * (X[3 * j + a] - xs[a]);
    }
    r->o = o;
    for (int a = 0; a < 3; ++a) r->go[a] = g[a] / (l * l);
    r->u = NAN;
    if (want_var) {
        forward_subst(L, N, kbuf, vbuf);
        double s = 0.0;
        for (int j = 0; j < N; ++j) s += vbuf[j] * vbuf[j];
        double u = 1.0 - s;
        r->u = u > 0.0 ? u : 0.0;
    }
    revert(P, r);
    if (!want_var) r->v = NAN;
}

static void eval_invalid(or_eval* r, int status) {
    r->o = NAN; r->u = NAN;
    r->go[0] = r->go[1] = r->go[2] = 0.0;
    r->d = INFINITY; r->gd[0] = r->gd[1] = r->gd[2] = 0.0; r->v = INFINITY;
    r->status = status;
}

/* ------------------------------------------------------------------------------------ */
/* batched independent instances                                                         */
/* ------------------------------------------------------------------------------------ */
int or_gp_batch(const or_params* P, int64_t n_inst, const int64_t* inst_off, const double* X,
                const int64_t* q_off, const double* Q, int want_var, double* d, double* grad,
                double* var, uint8_t* status, double* occ, double* grad_occ, double* u_out,
                double* alpha_out) {
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t I = 0; I < n_inst; ++I) {
        int N = (int)(inst_off[I + 1] - inst_off[I]);
        const double* XI = X + 3 * inst_off[I];
        double* L = (double*)malloc(sizeof(double) * ((int64_t)N * (N + 1) / 2 + 1));
        double* al = (double*)malloc(sizeof(double) * (N + 1));
        double* kb = (double*)malloc(sizeof(double) * (N + 1));
        double* vb = (double*)malloc(sizeof(double) * (N + 1));
        if (!L || !al || !kb || !vb) { err = 1; free(L); free(al); free(kb); free(vb); continue; }
        int ok = N > 0 && or_gp_fit(XI, N, P, L, al);
        if (alpha_out) for (int j = 0; j < N; ++j) alpha_out[inst_off[I] + j] = ok ? al[j] : NAN;
        for (int64_t q = q_off[I]; q < q_off[I + 1]; ++q) {
            or_eval r;
            const double* xs = Q + 3 * q;
            if (!(isfinite(xs[0]) && isfinite(xs[1]) && isfinite(xs[2]))) eval_invalid(&r, ST_BAD_INPUT);
            else if (N == 0) eval_invalid(&r, ST_NO_SUPPORT);
            else if (!ok) eval_invalid(&r, ST_FACTOR_FAIL);
            else gp_eval(XI, N, L, al, xs, P, want_var, kb, vb, &r);
            if (d) d[q] = r.d;
            if (grad) for (int a = 0; a < 3; ++a) grad[3 * q + a] = r.gd[a];
            if (var) var[q] = r.v;
            if (status) status[q] = (uint8_t)r.status;
            if (occ) occ[q] = r.o;
            if (grad_occ) for (int a = 0; a < 3; ++a) grad_occ[3 * q + a] = r.go[a];
            if (u_out) u_out[q] = r.u;
        }
        free(L); free(al); free(kb); free(vb);
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------------------ */
/* L-GPDF frame: voxelise, one GP per leaf, testing voxels, closest-node inference       */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t lkey;
    int32_t bit;
    int32_t pad;
    int64_t idx; /* input point index */
} vox_rec;

static int cmp_vox(const void* a, const void* b) {
    const vox_rec* x = (const vox_rec*)a;
    const vox_rec* y = (const vox_rec*)b;
    if (x->lkey != y->lkey) return x->lkey < y->lkey ? -1 : 1;
    if (x->bit != y->bit) return (x->bit > y->bit) - (x->bit < y->bit);
    return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct {
    or_params P;
    int64_t n_leaves;
    uint64_t* leaf_key;   /* sorted */
    int32_t* leaf_nocc;   /* occupied voxels before the cap */
    int64_t* inst_off;    /* [n_leaves + 1] */
    double* X;            /* training voxel centres, global FP64 */
    int64_t* L_off;       /* packed factor offsets */
    double* L;
    double* alpha;
    uint8_t* fit_ok;
    int64_t n_test;
    uint64_t* test_key;
    uint64_t* test_inst_key;
    double* test_d;
    double* test_v;
    double* test_grad;
    uint8_t* test_status;
    int8_t* test_sign;
    /* surface properties (Eq. 6), when given */
    int n_props;
    double* Y;            /* [T][n_props] voxel-mean property at each training point */
    double* Lc;           /* packed factors of K + sigma_prop^2 I */
    double* alpha_c;      /* [T][n_props] */
    uint8_t* fitc_ok;
    double* test_c;       /* [n_test][n_props] */
    double* test_w;       /* [n_test] */
} or_frame;

static void voxel_of_bit(const int64_t leaf[3], int bit, int64_t ijk[3]) {
    ijk[0] = 8 * leaf[0] + (bit & 7);
    ijk[1] = 8 * leaf[1] + ((bit >> 3) & 7);
    ijk[2] = 8 * leaf[2] + (bit >> 6);
}

void or_frame_free(or_frame* F) {
    if (!F) return;
    free(F->leaf_key); free(F->leaf_nocc); free(F->inst_off); free(F->X); free(F->L_off);
    free(F->L); free(F->alpha); free(F->fit_ok); free(F->test_key); free(F->test_inst_key);
    free(F->test_d); free(F->test_v); free(F->test_grad); free(F->test_status); free(F->test_sign);
    free(F->Y); free(F->Lc); free(F->alpha_c); free(F->fitc_ok); free(F->test_c); free(F->test_w);
    free(F);
}

/*
 * Testing points by ray casting from the sensor origin (Sec. IV-B).  The paper casts a ray from
 * the sensor origin to each surface voxel and queries the voxels on it that hold earlier
 * measurements, adds voxels along each surface voxel's normal, and signs the distance from
 * the sensor origin.  Readings taken here:
 *   - rays: the integer 3D Bresenham line from the origin's voxel to the surface voxel (the
 *     surface voxel itself excluded); a voxel on it is kept if it is in `known` (voxels of
 *     the global grid before this frame);
 *   - normal: smallest-eigenvalue eigenvector of the scatter of the occupied voxels in the
 *     3x3x3 block around the surface voxel (at least 3 of them), from the exact integer
 *     matrix n * sum(o o^T) - (sum o)(sum o)^T by cyclic Jacobi rotations in FP64, oriented
 *     towards the origin; voxels round(s + k n), k = +-1..+-K;
 *   - sign: + for surface voxels, ray voxels and k > 0, - for k < 0; a voxel reached with
 *     both signs is +.
 */
static void jacobi3(double a[3][3], double v[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v[i][j] = i == j ? 1.0 : 0.0;
    static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 12; ++sweep) {
        for (int r = 0; r < 3; ++r) {
            int p = PQ[r][0], q = PQ[r][1];
            if (a[p][q] == 0.0) continue;
            double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
            double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
            if (theta < 0.0) t = -t;
            double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
            for (int k = 0; k < 3; ++k) {
                double akp = a[k][p], akq = a[k][q];
                a[k][p] = c * akp - sn * akq;
                a[k][q] = sn * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                double apk = a[p][k], aqk = a[q][k];
                a[p][k] = c * apk - sn * aqk;
                a[q][k] = sn * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                double vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - sn * vkq;
                v[k][q] = sn * vkp + c * vkq;
            }
        }
    }
}

/* unit normal of surface voxel s (or 0 if fewer than 3 occupied voxels around it) */
static int voxel_normal(const uint64_t* occ, int64_t nocc, const int64_t s[3], double n[3]) {
    int64_t cnt = 0, S1[3] = {0, 0, 0}, S2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (find_key(occ, nocc, pack_key(s[0] + dx, s[1] + dy, s[2] + dz)) < 0) continue;
                int64_t o[3] = {dx, dy, dz};
                ++cnt;
                for (int a = 0; a < 3; ++a) {
                    S1[a] += o[a];
                    for (int b = 0; b < 3; ++b) S2[a][b] += o[a] * o[b];
                }
            }
    if (cnt < 3) return 0;
    double A[3][3], V[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) A[a][b] = (double)(cnt * S2[a][b] - S1[a] * S1[b]);
    jacobi3(A, V);
    int k = 0;
    for (int j = 1; j < 3; ++j) if (A[j][j] < A[k][k]) k = j;
    double nn = sqrt(V[0][k] * V[0][k] + V[1][k] * V[1][k] + V[2][k] * V[2][k]);
    for (int a = 0; a < 3; ++a) n[a] = V[a][k] / nn;
    return 1;
}

typedef struct {
    uint64_t key;
    int32_t sign;
    int32_t pad;
} ksign;

static int cmp_ksign(const void* a, const void* b) {
    const ksign* x = (const ksign*)a;
    const ksign* y = (const ksign*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->sign < y->sign) - (x->sign > y->sign); /* + first */
}

typedef struct {
    ksign* v;
    int64_t n, cap;
} kslist;

static void ks_push(kslist* L, int64_t x, int64_t y, int64_t z, int sign) {
    if (!(x > -IJK_LIMIT && x < IJK_LIMIT && y > -IJK_LIMIT && y < IJK_LIMIT && z > -IJK_LIMIT && z < IJK_LIMIT)) return;
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->v = (ksign*)realloc(L->v, sizeof(ksign) * L->cap);
    }
    L->v[L->n].key = pack_key(x, y, z);
    L->v[L->n].sign = sign;
    L->v[L->n].pad = 0;
    L->n++;
}

/* integer 3D Bresenham from a to b, b excluded */
static void bresenham(const int64_t a[3], const int64_t b[3], const uint64_t* known, int64_t nknown, kslist* L) {
    int64_t d[3], st[3], p[3] = {a[0], a[1], a[2]};
    for (int k = 0; k < 3; ++k) {
        d[k] = b[k] > a[k] ? b[k] - a[k] : a[k] - b[k];
        st[k] = b[k] > a[k] ? 1 : -1;
    }
    int m = 0;
    if (d[1] > d[m]) m = 1;
    if (d[2] > d[m]) m = 2;
    int u = (m + 1) % 3, w = (m + 2) % 3;
    int64_t eu = 2 * d[u] - d[m], ew = 2 * d[w] - d[m];
    for (int64_t i = 0; i < d[m]; ++i) {
        if (find_key(known, nknown, pack_key(p[0], p[1], p[2])) >= 0) ks_push(L, p[0], p[1], p[2], 1);
        if (eu > 0) { p[u] += st[u]; eu -= 2 * d[m]; }
        if (ew > 0) { p[w] += st[w]; ew -= 2 * d[m]; }
        eu += 2 * d[u];
        ew += 2 * d[w];
        p[m] += st[m];
    }
}

or_frame* or_frame_build3(const or_params* P, const float* pts, const float* props, int64_t n, const double* origin,
                          int normal_steps, const uint64_t* known, int64_t n_known);
or_frame* or_frame_build(const or_params* P, const float* pts, int64_t n) {
    return or_frame_build3(P, pts, NULL, n, NULL, 0, NULL, 0);
}
or_frame* or_frame_build2(const or_params* P, const float* pts, int64_t n, const double* origin, int normal_steps,
                          const uint64_t* known, int64_t n_known) {
    return or_frame_build3(P, pts, NULL, n, origin, normal_steps, known, n_known);
}

/* Surface-property GP of one leaf (Eq. 6): Lc = chol(K + sigma_prop^2 I), and for each
 * channel alpha_c = (K + sigma_prop^2 I)^-1 y_c.  Y and alpha_c are [N][nc]. */
static int gp_fit_props(const double* X, int N, const or_params* P, int nc, const double* Y, double* Lc,
                        double* alpha_c) {
    double s2 = P->sigma_prop * P->sigma_prop;
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < i; ++j) Lc[PK(i, j)] = se_kernel(X + 3 * i, X + 3 * j, P->lengthscale);
        Lc[PK(i, i)] = 1.0 + s2;
    }
    if (!cholesky_packed(Lc, N)) return 0;
    double* y = (double*)malloc(sizeof(double) * (N > 0 ? N : 1));
    double* z = (double*)malloc(sizeof(double) * (N > 0 ? N : 1));
    double* a = (double*)malloc(sizeof(double) * (N > 0 ? N : 1));
    for (int c = 0; c < nc; ++c) {
        for (int i = 0; i < N; ++i) y[i] = Y[(int64_t)i * nc + c];
        forward_subst(Lc, N, y, z);
        back_subst(Lc, N, z, a);
        for (int i = 0; i < N; ++i) alpha_c[(int64_t)i * nc + c] = a[i];
    }
    free(y); free(z); free(a);
    return 1;
}

/* Property mean c_c = k^T alpha_c (Eq. 6) and variance w = 1 - |Lc^-1 k|^2 (the posterior
 * variance read as for Eq. 2) at xs. */
static void gp_eval_props(const double* X, int N, const double* Lc, const double* alpha_c, int nc,
                          const double xs[3], double l, double* kbuf, double* vbuf, double* c_out, double* w_out) {
    for (int c = 0; c < nc; ++c) c_out[c] = 0.0;
    for (int j = 0; j < N; ++j) {
        double k = se_kernel(xs, X + 3 * j, l);
        kbuf[j] = k;
        for (int c = 0; c < nc; ++c) c_out[c] += alpha_c[(int64_t)j * nc + c] * k;
    }
    forward_subst(Lc, N, kbuf, vbuf);
    double s = 0.0;
    for (int j = 0; j < N; ++j) s += vbuf[j] * vbuf[j];
    double w = 1.0 - s;
    *w_out = w > 0.0 ? w : 0.0;
}

or_frame* or_frame_build3(const or_params* P, const float* pts, const float* props, int64_t n, const double* origin,
                          int normal_steps, const uint64_t* known, int64_t n_known) {
    or_frame* F = (or_frame*)calloc(1, sizeof(or_frame));
    if (!F) return NULL;
    F->P = *P;
    double vs = P->voxel_size;
    /* 1. voxelise: (leaf key, bit) of every valid point, then unique */
    vox_rec* R = (vox_rec*)malloc(sizeof(vox_rec) * (n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {(double)pts[3 * i], (double)pts[3 * i + 1], (double)pts[3 * i + 2]};
        int64_t ijk[3], leaf[3];
        int32_t bit;
        if (!voxel_ijk(p, vs, ijk)) continue;
        leaf_of(ijk, leaf, &bit);
        R[m].lkey = pack_key(leaf[0], leaf[1], leaf[2]);
        R[m].bit = bit;
        R[m].pad = 0;
        R[m].idx = i;
        ++m;
    }
    qsort(R, (size_t)m, sizeof(vox_rec), cmp_vox);
    /* unique voxels; with properties, each voxel's property is the mean over its points
     * (summed in FP64 in ascending point index) */
    const int nc = (props && P->n_props > 0) ? P->n_props : 0;
    double* vmean = nc ? (double*)calloc((size_t)(m + 1) * nc, sizeof(double)) : NULL;
    int64_t* vcnt = nc ? (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t)) : NULL;
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (u == 0 || R[i].lkey != R[u - 1].lkey || R[i].bit != R[u - 1].bit) R[u++] = R[i];
        if (nc) {
            for (int c = 0; c < nc; ++c) vmean[(u - 1) * nc + c] += (double)props[R[i].idx * nc + c];
            vcnt[u - 1]++;
        }
    }
    if (nc)
        for (int64_t i = 0; i < u; ++i)
            for (int c = 0; c < nc; ++c) vmean[i * nc + c] /= (double)vcnt[i];
    /* 2. leaves, occupied counts, capped training sets */
    int64_t nl = 0;
    for (int64_t i = 0; i < u; ++i) if (i == 0 || R[i].lkey != R[i - 1].lkey) ++nl;
    F->n_leaves = nl;
    F->leaf_key = (uint64_t*)malloc(sizeof(uint64_t) * (nl + 1));
    F->leaf_nocc = (int32_t*)malloc(sizeof(int32_t) * (nl + 1));
    F->inst_off = (int64_t*)malloc(sizeof(int64_t) * (nl + 1));
    int64_t* run_start = (int64_t*)malloc(sizeof(int64_t) * (nl + 1));
    {
        int64_t li = -1;
        for (int64_t i = 0; i < u; ++i) {
            if (i == 0 || R[i].lkey != R[i - 1].lkey) {
                ++li;
                F->leaf_key[li] = R[i].lkey;
                F->leaf_nocc[li] = 0;
                run_start[li] = i;
            }
            F->leaf_nocc[li]++;
        }
    }
    int cap = P->max_pts_leaf;
    F->inst_off[0] = 0;
    for (int64_t l = 0; l < nl; ++l) {
        int64_t N = F->leaf_nocc[l] > cap ? cap : F->leaf_nocc[l];
        F->inst_off[l + 1] = F->inst_off[l] + N;
    }
    int64_t T = F->inst_off[nl];
    F->X = (double*)malloc(sizeof(double) * 3 * (T + 1));
    F->L_off = (int64_t*)malloc(sizeof(int64_t) * (nl + 1));
    F->L_off[0] = 0;
    for (int64_t l = 0; l < nl; ++l) {
        int64_t N = F->inst_off[l + 1] - F->inst_off[l];
        F->L_off[l + 1] = F->L_off[l] + N * (N + 1) / 2;
    }
    F->L = (double*)malloc(sizeof(double) * (F->L_off[nl] + 1));
    F->alpha = (double*)malloc(sizeof(double) * (T + 1));
    F->fit_ok = (uint8_t*)malloc(nl + 1);
    F->n_props = nc;
    if (nc) {
        F->Y = (double*)malloc(sizeof(double) * (T + 1) * nc);
        F->Lc = (double*)malloc(sizeof(double) * (F->L_off[nl] + 1));
        F->alpha_c = (double*)malloc(sizeof(double) * (T + 1) * nc);
        F->fitc_ok = (uint8_t*)malloc(nl + 1);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t l = 0; l < nl; ++l) {
        int64_t nocc = F->leaf_nocc[l];
        int64_t N = F->inst_off[l + 1] - F->inst_off[l];
        int64_t leaf[3];
        unpack_key(F->leaf_key[l], leaf);
        for (int64_t k = 0; k < N; ++k) {
            int64_t pick = nocc > cap ? (k * nocc) / cap : k;
            int64_t ijk[3];
            voxel_of_bit(leaf, R[run_start[l] + pick].bit, ijk);
            for (int a = 0; a < 3; ++a) F->X[3 * (F->inst_off[l] + k) + a] = (double)ijk[a] * vs;
            for (int c = 0; c < nc; ++c) F->Y[(F->inst_off[l] + k) * nc + c] = vmean[(run_start[l] + pick) * nc + c];
        }
        F->fit_ok[l] = (uint8_t)or_gp_fit(F->X + 3 * F->inst_off[l], (int)N, P, F->L + F->L_off[l],
                                          F->alpha + F->inst_off[l]);
        if (nc)
            F->fitc_ok[l] = (uint8_t)gp_fit_props(F->X + 3 * F->inst_off[l], (int)N, P, nc, F->Y + F->inst_off[l] * nc,
                                                  F->Lc + F->L_off[l], F->alpha_c + F->inst_off[l] * nc);
    }
    free(run_start);
    free(vmean);
    free(vcnt);
    /* 3. testing voxels: the dilated GP leaves (no origin), or the ray-cast set (Sec. IV-B) */
    kslist TL = {NULL, 0, 0};
    if (!origin) {
        uint64_t* tl = (uint64_t*)malloc(sizeof(uint64_t) * (27 * nl + 1));
        int64_t ntl = 0;
        for (int64_t l = 0; l < nl; ++l) {
            int64_t leaf[3];
            unpack_key(F->leaf_key[l], leaf);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) tl[ntl++] = pack_key(leaf[0] + dx, leaf[1] + dy, leaf[2] + dz);
        }
        qsort(tl, (size_t)ntl, sizeof(uint64_t), cmp_u64);
        int64_t ut = 0;
        for (int64_t i = 0; i < ntl; ++i) if (ut == 0 || tl[i] != tl[ut - 1]) tl[ut++] = tl[i];
        for (int64_t t = 0; t < ut; ++t) {
            int64_t M[3];
            unpack_key(tl[t], M);
            for (int b = 0; b < 512; ++b) {
                int64_t ijk[3];
                voxel_of_bit(M, b, ijk);
                ks_push(&TL, ijk[0], ijk[1], ijk[2], 1);
            }
        }
        free(tl);
    } else {
        /* occupied voxels of this frame, sorted */
        uint64_t* occ = (uint64_t*)malloc(sizeof(uint64_t) * (u + 1));
        for (int64_t i = 0; i < u; ++i) {
            int64_t leaf[3], ijk[3];
            unpack_key(R[i].lkey, leaf);
            voxel_of_bit(leaf, R[i].bit, ijk);
            occ[i] = pack_key(ijk[0], ijk[1], ijk[2]);
        }
        qsort(occ, (size_t)u, sizeof(uint64_t), cmp_u64);
        int64_t ov[3];
        int have_o = voxel_ijk(origin, vs, ov);
        for (int64_t i = 0; i < u; ++i) {
            int64_t sv[3];
            unpack_key(occ[i], sv);
            ks_push(&TL, sv[0], sv[1], sv[2], 1);
            double nrm[3];
            if (have_o && voxel_normal(occ, u, sv, nrm)) {
                double e = 0.0;
                for (int a = 0; a < 3; ++a) e += nrm[a] * (origin[a] - (double)sv[a] * vs);
                if (e < 0.0) for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
                for (int k = -normal_steps; k <= normal_steps; ++k) {
                    if (k == 0) continue;
                    int64_t v[3];
                    for (int a = 0; a < 3; ++a) v[a] = sv[a] + (int64_t)floor((double)k * nrm[a] + 0.5);
                    ks_push(&TL, v[0], v[1], v[2], k > 0 ? 1 : -1);
                }
            }
            if (have_o) bresenham(ov, sv, known, n_known, &TL);
        }
        free(occ);
    }
    qsort(TL.v, (size_t)TL.n, sizeof(ksign), cmp_ksign);
    int64_t nt = 0;
    for (int64_t i = 0; i < TL.n; ++i)
        if (nt == 0 || TL.v[i].key != TL.v[nt - 1].key) TL.v[nt++] = TL.v[i];  /* + sorts first */
    free(R);
    F->n_test = nt;
    F->test_key = (uint64_t*)malloc(sizeof(uint64_t) * (F->n_test + 1));
    F->test_inst_key = (uint64_t*)malloc(sizeof(uint64_t) * (F->n_test + 1));
    F->test_d = (double*)malloc(sizeof(double) * (F->n_test + 1));
    F->test_v = (double*)malloc(sizeof(double) * (F->n_test + 1));
    F->test_grad = (double*)malloc(sizeof(double) * 3 * (F->n_test + 1));
    F->test_status = (uint8_t*)malloc(F->n_test + 1);
    F->test_sign = (int8_t*)malloc(F->n_test + 1);
    if (nc) {
        F->test_c = (double*)malloc(sizeof(double) * (F->n_test + 1) * nc);
        F->test_w = (double*)malloc(sizeof(double) * (F->n_test + 1));
    }
    int Nmax = 1;
    for (int64_t l = 0; l < nl; ++l) {
        int64_t N = F->inst_off[l + 1] - F->inst_off[l];
        if (N > Nmax) Nmax = (int)N;
    }
    /* 4. closest GP node per testing voxel, inference, sign */
#pragma omp parallel
    {
        double* kb = (double*)malloc(sizeof(double) * Nmax);
        double* vb = (double*)malloc(sizeof(double) * Nmax);
#pragma omp for schedule(dynamic, 256)
        for (int64_t o = 0; o < nt; ++o) {
            int64_t ijk[3], M[3];
            int32_t bit;
            unpack_key(TL.v[o].key, ijk);
            leaf_of(ijk, M, &bit);
            int64_t inst = find_key(F->leaf_key, nl, pack_key(M[0], M[1], M[2]));
            if (inst < 0) {
                int64_t best_d2 = INT64_MAX;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (!dx && !dy && !dz) continue;
                            int64_t Fl[3] = {M[0] + dx, M[1] + dy, M[2] + dz};
                            int64_t f = find_key(F->leaf_key, nl, pack_key(Fl[0], Fl[1], Fl[2]));
                            if (f < 0) continue;
                            int64_t d2 = 0;
                            for (int a = 0; a < 3; ++a) {
                                int64_t e = 2 * ijk[a] - (16 * Fl[a] + 7);
                                d2 += e * e;
                            }
                            if (d2 < best_d2) { best_d2 = d2; inst = f; }
                        }
            }
            if (inst < 0) { /* beyond the 26 neighbours: nearest GP leaf within the search radius */
                int Rr = P->max_leaf_search;
                int64_t best_d2 = INT64_MAX;
                uint64_t best_key = 0;
                for (int dz = -Rr; dz <= Rr; ++dz)
                    for (int dy = -Rr; dy <= Rr; ++dy)
                        for (int dx = -Rr; dx <= Rr; ++dx) {
                            int64_t Fl[3] = {M[0] + dx, M[1] + dy, M[2] + dz};
                            uint64_t k = pack_key(Fl[0], Fl[1], Fl[2]);
                            int64_t f = find_key(F->leaf_key, nl, k);
                            if (f < 0) continue;
                            int64_t d2 = 0;
                            for (int a = 0; a < 3; ++a) {
                                int64_t e = 2 * ijk[a] - (16 * Fl[a] + 7);
                                d2 += e * e;
                            }
                            if (d2 < best_d2 || (d2 == best_d2 && k < best_key)) { best_d2 = d2; best_key = k; inst = f; }
                        }
            }
            F->test_key[o] = TL.v[o].key;
            F->test_sign[o] = (int8_t)TL.v[o].sign;
            or_eval r;
            double xs[3] = {(double)ijk[0] * vs, (double)ijk[1] * vs, (double)ijk[2] * vs};
            if (inst < 0) {
                eval_invalid(&r, ST_NO_SUPPORT);
                F->test_inst_key[o] = 0;
            } else {
                F->test_inst_key[o] = F->leaf_key[inst];
                int N = (int)(F->inst_off[inst + 1] - F->inst_off[inst]);
                if (!F->fit_ok[inst]) eval_invalid(&r, ST_FACTOR_FAIL);
                else gp_eval(F->X + 3 * F->inst_off[inst], N, F->L + F->L_off[inst], F->alpha + F->inst_off[inst], xs,
                             P, 1, kb, vb, &r);
            }
            double sg = (double)TL.v[o].sign;
            F->test_d[o] = r.status == ST_OK || r.status == ST_CLAMPED ? sg * r.d : r.d;
            F->test_v[o] = r.v;
            for (int a = 0; a < 3; ++a) F->test_grad[3 * o + a] = sg * r.gd[a];
            F->test_status[o] = (uint8_t)r.status;
            if (nc) {
                if (inst < 0 || !F->fitc_ok[inst]) {
                    for (int c = 0; c < nc; ++c) F->test_c[o * nc + c] = NAN;
                    F->test_w[o] = INFINITY;
                } else {
                    int N = (int)(F->inst_off[inst + 1] - F->inst_off[inst]);
                    gp_eval_props(F->X + 3 * F->inst_off[inst], N, F->Lc + F->L_off[inst],
                                  F->alpha_c + F->inst_off[inst] * nc, nc, xs, P->lengthscale, kb, vb,
                                  F->test_c + o * nc, F->test_w + o);
                }
            }
        }
        free(kb);
        free(vb);
    }
    free(TL.v);
    return F;
}


int64_t or_frame_count(const or_frame* F, int what) {
    if (what == 0) return F->n_leaves;
    if (what == 1) return F->inst_off[F->n_leaves];
    if (what == 2) return F->n_test;
    return -1;
}

void or_frame_leaves(const or_frame* F, uint64_t* key, int32_t* nocc, int64_t* inst_off,
                     double* X, double* alpha) {
    int64_t nl = F->n_leaves, T = F->inst_off[nl];
    if (key) memcpy(key, F->leaf_key, sizeof(uint64_t) * nl);
    if (nocc) memcpy(nocc, F->leaf_nocc, sizeof(int32_t) * nl);
    if (inst_off) memcpy(inst_off, F->inst_off, sizeof(int64_t) * (nl + 1));
    if (X) memcpy(X, F->X, sizeof(double) * 3 * T);
    if (alpha) memcpy(alpha, F->alpha, sizeof(double) * T);
}

/* property means [n_test][n_props] and variances [n_test]; returns n_props (0: none) */
int or_frame_props(const or_frame* F, double* c, double* w) {
    if (!F->n_props) return 0;
    if (c) memcpy(c, F->test_c, sizeof(double) * F->n_test * F->n_props);
    if (w) memcpy(w, F->test_w, sizeof(double) * F->n_test);
    return F->n_props;
}

void or_frame_signs(const or_frame* F, int8_t* sign) {
    if (sign) memcpy(sign, F->test_sign, F->n_test);
}

void or_frame_tests(const or_frame* F, uint64_t* key, uint64_t* inst_key, double* d, double* v,
                    double* grad, uint8_t* status) {
    int64_t n = F->n_test;
    if (key) memcpy(key, F->test_key, sizeof(uint64_t) * n);
    if (inst_key) memcpy(inst_key, F->test_inst_key, sizeof(uint64_t) * n);
    if (d) memcpy(d, F->test_d, sizeof(double) * n);
    if (v) memcpy(v, F->test_v, sizeof(double) * n);
    if (grad) memcpy(grad, F->test_grad, sizeof(double) * 3 * n);
    if (status) memcpy(status, F->test_status, n);
}

/* ------------------------------------------------------------------------------------ */
/* global grid + probabilistic fusion (Eqs. 7-9)                                        */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    double D, V;
    double C[MAX_PROPS]; /* fused surface properties; W = NaN: none fused yet */
    double W;
} gvox;

typedef struct {
    int64_t n;
    gvox* v;       /* sorted by key */
    int64_t nl;
    uint64_t* lkey; /* sorted */
    uint8_t* lflag; /* bit0: touched by the latest fuse; bit1: ever touched */
    int n_props;
} or_grid;

or_grid* or_grid_new(void) { return (or_grid*)calloc(1, sizeof(or_grid)); }

void or_grid_free(or_grid* g) {
    if (!g) return;
    free(g->v); free(g->lkey); free(g->lflag); free(g);
}

typedef struct {
    uint64_t key;
    double d, v;
    int64_t order;
    double c[MAX_PROPS], w;
    int hasp;
} fin;

static int cmp_fin(const void* a, const void* b) {
    const fin* x = (const fin*)a;
    const fin* y = (const fin*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->order > y->order) - (x->order < y->order);
}

static uint64_t leaf_key_of_voxel_key(uint64_t vk) {
    int64_t ijk[3];
    unpack_key(vk, ijk);
    return pack_key(floor_div8(ijk[0]), floor_div8(ijk[1]), floor_div8(ijk[2]));
}

/* one fusion step of a stored voxel (D, V) with a new estimate (d, v) */
static void fuse_one(int mode, double* D, double* V, double d, double v) {
    if (mode == 0) { /* Eqs. 7-8 */
        double Vp = *V;
        double a = Vp / (Vp + v);
        double b = v / (Vp + v);
        *D = a * d + b * (*D);
        *V = 1.0 / (1.0 / Vp + 1.0 / v);
    } else { /* Eq. 9: V is the accumulated weight, the new weight is 1 - v */
        double Vp = *V, w = 1.0 - v;
        double a = w / (Vp + w);
        double b = Vp / (Vp + w);
        *D = a * d + b * (*D);
        *V = Vp + w;
    }
}

/* Surface-property fusion (the last sentence of Sec. IV-C): the rules of fuse_one applied to
 * every channel of C with the shared variance (or weight) W and the new variance w. */
static void fuse_props(int mode, double* C, double* W, const double* c, double w, int nc) {
    if (isnan(*W)) {
        for (int k = 0; k < nc; ++k) C[k] = c[k];
        *W = mode == 0 ? w : 1.0 - w;
        return;
    }
    if (mode == 0) {
        double Wp = *W;
        double a = Wp / (Wp + w);
        double b = w / (Wp + w);
        for (int k = 0; k < nc; ++k) C[k] = a * c[k] + b * C[k];
        *W = 1.0 / (1.0 / Wp + 1.0 / w);
    } else {
        double Wp = *W, ww = 1.0 - w;
        double a = ww / (Wp + ww);
        double b = Wp / (Wp + ww);
        for (int k = 0; k < nc; ++k) C[k] = a * c[k] + b * C[k];
        *W = Wp + ww;
    }
}

int or_grid_fuse2(or_grid* g, int mode, const uint64_t* key, const double* d, const double* v,
                  const uint8_t* status, const double* c, const double* w, int nc, int64_t n);

int or_grid_fuse(or_grid* g, int mode, const uint64_t* key, const double* d, const double* v,
                 const uint8_t* status, int64_t n) {
    return or_grid_fuse2(g, mode, key, d, v, status, NULL, NULL, 0, n);
}

/* Fusion of one frame's testing voxels; with c / w (nc channels) the surface properties of
 * the voxels whose distance is fused are fused too, when every channel is finite and w is a
 * valid variance (finite, > 0, and < 1 for Eq. 9). */
int or_grid_fuse2(or_grid* g, int mode, const uint64_t* key, const double* d, const double* v,
                  const uint8_t* status, const double* c, const double* w, int nc, int64_t n) {
    if (nc < 0 || nc > MAX_PROPS) return -1;
    if (!c || !w) nc = 0;
    if (nc > g->n_props) g->n_props = nc;
    fin* in = (fin*)malloc(sizeof(fin) * (n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (status[i] != ST_OK || !isfinite(d[i]) || !isfinite(v[i]) || !(v[i] > 0.0)) continue;
        if (mode == 1 && !(v[i] < 1.0)) continue;
        in[m].key = key[i]; in[m].d = d[i]; in[m].v = v[i]; in[m].order = i;
        in[m].hasp = 0;
        if (nc) {
            int ok = isfinite(w[i]) && w[i] > 0.0 && (mode == 0 || w[i] < 1.0);
            for (int k = 0; k < nc; ++k) {
                in[m].c[k] = c[i * nc + k];
                if (!isfinite(in[m].c[k])) ok = 0;
            }
            in[m].w = w[i];
            in[m].hasp = ok;
        }
        ++m;
    }
    qsort(in, (size_t)m, sizeof(fin), cmp_fin);
    gvox* out = (gvox*)malloc(sizeof(gvox) * (g->n + m + 1));
    int64_t a = 0, b = 0, o = 0;
    while (a < g->n || b < m) {
        if (b >= m || (a < g->n && g->v[a].key < in[b].key)) { out[o++] = g->v[a++]; continue; }
        gvox cur;
        if (a < g->n && g->v[a].key == in[b].key) cur = g->v[a++];
        else {
            cur.key = in[b].key;
            cur.D = in[b].d;
            cur.V = mode == 0 ? in[b].v : 1.0 - in[b].v;
            for (int k = 0; k < MAX_PROPS; ++k) cur.C[k] = NAN;
            cur.W = NAN;
            if (in[b].hasp) fuse_props(mode, cur.C, &cur.W, in[b].c, in[b].w, nc);
            ++b;
        }
        while (b < m && in[b].key == cur.key) {
            fuse_one(mode, &cur.D, &cur.V, in[b].d, in[b].v);
            if (in[b].hasp) fuse_props(mode, cur.C, &cur.W, in[b].c, in[b].w, nc);
            ++b;
        }
        out[o++] = cur;
    }
    free(g->v);
    g->v = out;
    g->n = o;
    /* leaf flags */
    for (int64_t i = 0; i < g->nl; ++i) g->lflag[i] &= (uint8_t)~1u;
    uint64_t* tk = (uint64_t*)malloc(sizeof(uint64_t) * (m + 1));
    int64_t nt = 0;
    for (int64_t i = 0; i < m; ++i) tk[nt++] = leaf_key_of_voxel_key(in[i].key);
    qsort(tk, (size_t)nt, sizeof(uint64_t), cmp_u64);
    int64_t ut = 0;
    for (int64_t i = 0; i < nt; ++i) if (ut == 0 || tk[i] != tk[ut - 1]) tk[ut++] = tk[i];
    uint64_t* nk = (uint64_t*)malloc(sizeof(uint64_t) * (g->nl + ut + 1));
    uint8_t* nf = (uint8_t*)malloc(g->nl + ut + 1);
    a = 0; b = 0; o = 0;
    while (a < g->nl || b < ut) {
        if (b >= ut || (a < g->nl && g->lkey[a] < tk[b])) { nk[o] = g->lkey[a]; nf[o++] = g->lflag[a++]; continue; }
        uint8_t f = 0;
        if (a < g->nl && g->lkey[a] == tk[b]) f = g->lflag[a++];
        nk[o] = tk[b++];
        nf[o++] = (uint8_t)(f | 3u);
    }
    free(g->lkey); free(g->lflag);
    g->lkey = nk; g->lflag = nf; g->nl = o;
    free(tk);
    free(in);
    return 0;
}

int64_t or_grid_size(const or_grid* g) { return g->n; }

/* fused properties [n][n_props] and their variances (weights for Eq. 9) in key order;
 * returns n_props */
int or_grid_export_props(const or_grid* g, double* C, double* W) {
    for (int64_t i = 0; i < g->n; ++i) {
        if (C) for (int k = 0; k < g->n_props; ++k) C[i * g->n_props + k] = g->v[i].C[k];
        if (W) W[i] = g->v[i].W;
    }
    return g->n_props;
}

void or_grid_export(const or_grid* g, uint64_t* key, double* D, double* V, uint8_t* flags) {
    for (int64_t i = 0; i < g->n; ++i) {
        if (key) key[i] = g->v[i].key;
        if (D) D[i] = g->v[i].D;
        if (V) V[i] = g->v[i].V;
        if (flags) {
            int64_t l = find_key(g->lkey, g->nl, leaf_key_of_voxel_key(g->v[i].key));
            flags[i] = l >= 0 ? g->lflag[l] : 0;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* zero crossings and marching cubes over the fused grid (Sec. IV-D)                     */
/*                                                                                      */
/* The fused values D live at voxel centres c(ijk) = ijk * vs.  A voxel is inside when   */
/* D < 0.  Each axis edge between two known neighbouring voxels a and b = a + e_axis     */
/* whose insides differ carries one zero crossing, placed by linear interpolation from   */
/* the lower end a: t = D_a / (D_a - D_b), p_axis = (a_axis + t) vs, the other two        */
/* coordinates a_k vs.  As a G-GPDF training point the crossing is rounded to float32;   */
/* it belongs to the voxel that float32 point falls in (always a or b), and so to that   */
/* voxel's leaf.  Marching cubes runs on the cells whose lower corner lies in a selected */
/* leaf and whose 8 corners are all known; each cell's polygon loops come from walking   */
/* its six faces, where every in->out edge (counter-clockwise seen from outside) is      */
/* joined to the out->in edge that closes the run of inside corners behind it, so inside */
/* corners that only touch diagonally stay apart.  The loops are fanned from their       */
/* lowest local edge and oriented so that triangle normals point to increasing D.        */
/* ------------------------------------------------------------------------------------ */
static const gvox* grid_find(const or_grid* g, const int64_t ijk[3]) {
    for (int a = 0; a < 3; ++a)
        if (ijk[a] <= -KEY_BIAS || ijk[a] >= KEY_BIAS) return NULL;
    uint64_t k = pack_key(ijk[0], ijk[1], ijk[2]);
    int64_t lo = 0, hi = g->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->v[mid].key < k) lo = mid + 1; else hi = mid;
    }
    return (lo < g->n && g->v[lo].key == k) ? &g->v[lo] : NULL;
}

static int leaf_selected(const or_grid* g, uint64_t leaf_key, int active_only) {
    int64_t l = find_key(g->lkey, g->nl, leaf_key);
    if (l < 0) return 0;
    return active_only ? (g->lflag[l] & 1) : 1;
}

/* the crossing on the edge from voxel a along `axis`, in FP64 */
static void crossing_point(const int64_t a[3], int axis, double Da, double Db, double vs, double p[3]) {
    double t = Da / (Da - Db);
    for (int k = 0; k < 3; ++k) p[k] = (double)a[k] * vs;
    p[axis] = ((double)a[axis] + t) * vs;
}

typedef struct {
    uint64_t leaf;
    int32_t bit, slot;
    float p[3];
    uint64_t owner;
    double c[MAX_PROPS];
} xrec;

/* property at a crossing: the fused properties of the two ends interpolated with the same t
 * (NaN unless both ends carry properties) */
static void crossing_props(const gvox* lo, const gvox* hi, int nc, double* out) {
    double t = lo->D / (lo->D - hi->D);
    for (int k = 0; k < nc; ++k)
        out[k] = (isnan(lo->W) || isnan(hi->W)) ? NAN : lo->C[k] + t * (hi->C[k] - lo->C[k]);
}

static int cmp_xrec(const void* a, const void* b) {
    const xrec* x = (const xrec*)a;
    const xrec* y = (const xrec*)b;
    if (x->leaf != y->leaf) return x->leaf < y->leaf ? -1 : 1;
    if (x->bit != y->bit) return x->bit < y->bit ? -1 : 1;
    return (x->slot > y->slot) - (x->slot < y->slot);
}

/* Zero crossings owned by the voxels of the selected leaves (all leaves, or those
 * touched by the latest fusion), ordered by leaf key, then in-leaf voxel bit, then
 * slot = 2 axis + (neighbour on the + side).  Returns the count; fills the outputs when
 * they are given (xyz: 3 floats per crossing). */
int64_t or_grid_crossings(const or_grid* g, double vs, int active_only, float* xyz, uint64_t* owner,
                          uint8_t* slot, double* cprop) {
    const int nc = g->n_props;
    int64_t cap = 16, m = 0;
    xrec* R = (xrec*)malloc(sizeof(xrec) * cap);
    for (int64_t i = 0; i < g->n; ++i) {
        int64_t v[3], leaf[3];
        int32_t bit;
        unpack_key(g->v[i].key, v);
        leaf_of(v, leaf, &bit);
        uint64_t lk = pack_key(leaf[0], leaf[1], leaf[2]);
        if (!leaf_selected(g, lk, active_only)) continue;
        for (int s = 0; s < 6; ++s) {
            int axis = s / 2, dir = (s & 1) ? 1 : -1;
            int64_t nb[3] = {v[0], v[1], v[2]};
            nb[axis] += dir;
            const gvox* o = grid_find(g, nb);
            if (!o) continue;
            const gvox *lo = dir > 0 ? &g->v[i] : o, *hi = dir > 0 ? o : &g->v[i];
            if ((lo->D < 0.0) == (hi->D < 0.0)) continue;
            int64_t a[3] = {v[0], v[1], v[2]};
            if (dir < 0) a[axis] -= 1;
            double p[3];
            crossing_point(a, axis, lo->D, hi->D, vs, p);
            float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
            double pd[3] = {(double)pf[0], (double)pf[1], (double)pf[2]};
            int64_t w[3];
            if (!voxel_ijk(pd, vs, w) || w[0] != v[0] || w[1] != v[1] || w[2] != v[2]) continue;
            if (m == cap) { cap *= 2; R = (xrec*)realloc(R, sizeof(xrec) * cap); }
            R[m].leaf = lk; R[m].bit = bit; R[m].slot = s;
            R[m].p[0] = pf[0]; R[m].p[1] = pf[1]; R[m].p[2] = pf[2];
            R[m].owner = g->v[i].key;
            crossing_props(lo, hi, nc, R[m].c);
            ++m;
        }
    }
    qsort(R, (size_t)m, sizeof(xrec), cmp_xrec);
    for (int64_t i = 0; i < m; ++i) {
        if (xyz) { xyz[3 * i] = R[i].p[0]; xyz[3 * i + 1] = R[i].p[1]; xyz[3 * i + 2] = R[i].p[2]; }
        if (owner) owner[i] = R[i].owner;
        if (slot) slot[i] = (uint8_t)R[i].slot;
        if (cprop) for (int k = 0; k < nc; ++k) cprop[i * nc + k] = R[i].c[k];
    }
    free(R);
    return m;
}

/* corners of the face with outward normal (2 side - 1) e_axis, counter-clockwise seen
 * from outside; corner index = x + 2 y + 4 z of the cell-local offset */
static void face_corners(int axis, int side, int q[4]) {
    static const int cyc[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}}; /* CCW in (u, w) seen from +axis */
    int u = (axis + 1) % 3, w = (axis + 2) % 3;                   /* e_u x e_w = e_axis */
    for (int i = 0; i < 4; ++i) {
        int j = side ? i : (4 - i) % 4;
        int c[3];
        c[axis] = side; c[u] = cyc[j][0]; c[w] = cyc[j][1];
        q[i] = c[0] + 2 * c[1] + 4 * c[2];
    }
}

/* cell-local edge between corners c0, c1 (differing in one bit): 3 * lower corner + axis */
static int cell_edge(int c0, int c1) {
    int x = c0 ^ c1, axis = x == 1 ? 0 : (x == 2 ? 1 : 2);
    int lo = c0 < c1 ? c0 : c1;
    return 3 * lo + axis;
}

/* Triangles of one cell from its inside mask; out[3 t + j] are cell-local edges
 * (3 * lower corner + axis).  Returns the triangle count. */
static int cell_triangles(int inside_mask, int* out) {
    int next[24];
    for (int e = 0; e < 24; ++e) next[e] = -1;
    for (int axis = 0; axis < 3; ++axis)
        for (int side = 0; side < 2; ++side) {
            int q[4];
            face_corners(axis, side, q);
            for (int k = 0; k < 4; ++k) {
                int ck = q[k], cn = q[(k + 1) % 4];
                if (!((inside_mask >> ck) & 1) || ((inside_mask >> cn) & 1)) continue;
                int j = k;
                while ((inside_mask >> q[(j + 3) % 4]) & 1) j = (j + 3) % 4;
                next[cell_edge(ck, cn)] = cell_edge(q[(j + 3) % 4], q[j]);
            }
        }
    int seen[24] = {0}, nt = 0;
    for (int e = 0; e < 24; ++e) {
        if (next[e] < 0 || seen[e]) continue;
        int loop[24], m = 0;
        for (int f = e; !seen[f]; f = next[f]) { seen[f] = 1; loop[m++] = f; }
        /* the face walk runs the loop with normals toward the inside: fan it reversed */
        for (int i = 1; i + 1 < m; ++i) {
            out[3 * nt] = loop[0];
            out[3 * nt + 1] = loop[i + 1];
            out[3 * nt + 2] = loop[i];
            ++nt;
        }
    }
    return nt;
}

/* Marching-cubes triangles of the cells whose lower corner lies in a selected leaf and
 * whose 8 corners are known.  Per triangle: xyz 9 doubles (FP64 crossing points), and
 * for each vertex its edge as (key of the edge's lower voxel, axis).  Cells in ascending
 * key order of the lower corner, triangles in fan order.  Returns the triangle count. */
int64_t or_grid_mesh(const or_grid* g, double vs, int active_only, double* xyz, uint64_t* ekey, uint8_t* eaxis,
                     double* vprop) {
    const int nc = g->n_props;
    int64_t nt = 0;
    for (int64_t i = 0; i < g->n; ++i) {
        int64_t v[3], leaf[3];
        int32_t bit;
        unpack_key(g->v[i].key, v);
        leaf_of(v, leaf, &bit);
        if (!leaf_selected(g, pack_key(leaf[0], leaf[1], leaf[2]), active_only)) continue;
        double D[8];
        const gvox* corner[8];
        int mask = 0, ok = 1;
        for (int c = 0; c < 8 && ok; ++c) {
            int64_t w[3] = {v[0] + (c & 1), v[1] + ((c >> 1) & 1), v[2] + ((c >> 2) & 1)};
            const gvox* o = grid_find(g, w);
            if (!o) { ok = 0; break; }
            corner[c] = o;
            D[c] = o->D;
            if (D[c] < 0.0) mask |= 1 << c;
        }
        if (!ok || mask == 0 || mask == 255) continue;
        int tri[3 * 24];
        int n = cell_triangles(mask, tri);
        for (int t = 0; t < n; ++t, ++nt) {
            for (int j = 0; j < 3; ++j) {
                int e = tri[3 * t + j], lc = e / 3, axis = e % 3;
                int64_t a[3] = {v[0] + (lc & 1), v[1] + ((lc >> 1) & 1), v[2] + ((lc >> 2) & 1)};
                int uc = lc | (1 << axis);
                double p[3];
                crossing_point(a, axis, D[lc], D[uc], vs, p);
                if (xyz) for (int k = 0; k < 3; ++k) xyz[9 * nt + 3 * j + k] = p[k];
                if (ekey) ekey[3 * nt + j] = pack_key(a[0], a[1], a[2]);
                if (eaxis) eaxis[3 * nt + j] = (uint8_t)axis;
                if (vprop && nc) crossing_props(corner[lc], corner[uc], nc, vprop + (3 * nt + j) * nc);
            }
        }
    }
    return nt;
}

/* ------------------------------------------------------------------------------------ */
/* G-GPDF: surface points binned by leaf; per-neighbourhood GPs for arbitrary queries    */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    or_params P;
    int64_t n_pts;
    double* pts;      /* widened input, n_pts*3 */
    int64_t nl;
    uint64_t* lkey;   /* sorted occupied leaves */
    int64_t* off;     /* [nl + 1] */
    int64_t* idx;     /* point indices, ascending within a leaf */
} or_surface;

typedef struct {
    uint64_t k;
    int64_t i;
} kidx;

static int cmp_kidx(const void* a, const void* b) {
    const kidx* x = (const kidx*)a;
    const kidx* y = (const kidx*)b;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    return (x->i > y->i) - (x->i < y->i);
}

void or_surface_free(or_surface* S) {
    if (!S) return;
    free(S->pts); free(S->lkey); free(S->off); free(S->idx); free(S);
}

or_surface* or_surface_new(const or_params* P, const float* pts, int64_t n) {
    or_surface* S = (or_surface*)calloc(1, sizeof(or_surface));
    S->P = *P;
    S->n_pts = n;
    S->pts = (double*)malloc(sizeof(double) * 3 * (n + 1));
    kidx* R = (kidx*)malloc(sizeof(kidx) * (n + 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) S->pts[3 * i + a] = (double)pts[3 * i + a];
        int64_t ijk[3], leaf[3];
        int32_t bit;
        if (!voxel_ijk(S->pts + 3 * i, P->voxel_size, ijk)) continue;
        leaf_of(ijk, leaf, &bit);
        R[m].k = pack_key(leaf[0], leaf[1], leaf[2]);
        R[m].i = i;
        ++m;
    }
    qsort(R, (size_t)m, sizeof(kidx), cmp_kidx);
    int64_t nl = 0;
    for (int64_t i = 0; i < m; ++i) if (i == 0 || R[i].k != R[i - 1].k) ++nl;
    S->nl = nl;
    S->lkey = (uint64_t*)malloc(sizeof(uint64_t) * (nl + 1));
    S->off = (int64_t*)malloc(sizeof(int64_t) * (nl + 1));
    S->idx = (int64_t*)malloc(sizeof(int64_t) * (m + 1));
    int64_t l = -1;
    for (int64_t i = 0; i < m; ++i) {
        if (i == 0 || R[i].k != R[i - 1].k) { ++l; S->lkey[l] = R[i].k; S->off[l] = i; }
        S->idx[i] = R[i].i;
    }
    S->off[nl] = m;
    free(R);
    return S;
}

int64_t or_surface_leaves(const or_surface* S, uint64_t* key, int64_t* off, int64_t* idx) {
    if (key) memcpy(key, S->lkey, sizeof(uint64_t) * S->nl);
    if (off) memcpy(off, S->off, sizeof(int64_t) * (S->nl + 1));
    if (idx) memcpy(idx, S->idx, sizeof(int64_t) * S->off[S->nl]);
    return S->nl;
}

/* Centre leaf of the instance that serves query leaf M, or -1 (status 1). */
static int centre_leaf(const or_surface* S, const int64_t M[3], int64_t C[3]) {
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                if (find_key(S->lkey, S->nl, pack_key(M[0] + dx, M[1] + dy, M[2] + dz)) >= 0) {
                    C[0] = M[0]; C[1] = M[1]; C[2] = M[2];
                    return 1;
                }
    int R = S->P.max_leaf_search;
    int64_t best_d2 = INT64_MAX;
    uint64_t best_key = 0;
    int found = 0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                uint64_t k = pack_key(M[0] + dx, M[1] + dy, M[2] + dz);
                if (find_key(S->lkey, S->nl, k) < 0) continue;
                int64_t d2 = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
                if (!found || d2 < best_d2 || (d2 == best_d2 && k < best_key)) {
                    found = 1; best_d2 = d2; best_key = k;
                }
            }
    if (!found) return 0;
    unpack_key(best_key, C);
    return 1;
}

typedef struct {
    double d2;
    int64_t i;
} didx;

static int cmp_didx(const void* a, const void* b) {
    const didx* x = (const didx*)a;
    const didx* y = (const didx*)b;
    if (x->d2 != y->d2) return x->d2 < y->d2 ? -1 : 1;
    return (x->i > y->i) - (x->i < y->i);
}

/* Point indices of the instance centred on leaf C (27 leaves, capped, ascending index). */
int64_t or_surface_instance(const or_surface* S, uint64_t ckey, int64_t* out_idx) {
    int64_t C[3];
    unpack_key(ckey, C);
    int64_t cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t l = find_key(S->lkey, S->nl, pack_key(C[0] + dx, C[1] + dy, C[2] + dz));
                if (l >= 0) cnt += S->off[l + 1] - S->off[l];
            }
    didx* cand = (didx*)malloc(sizeof(didx) * (cnt + 1));
    int64_t m = 0;
    double vs = S->P.voxel_size;
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = ((double)(8 * C[a]) + 3.5) * vs;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t l = find_key(S->lkey, S->nl, pack_key(C[0] + dx, C[1] + dy, C[2] + dz));
                if (l < 0) continue;
                for (int64_t t = S->off[l]; t < S->off[l + 1]; ++t) {
                    int64_t i = S->idx[t];
                    const double* x = S->pts + 3 * i;
                    double ex = x[0] - c[0], ey = x[1] - c[1], ez = x[2] - c[2];
                    cand[m].d2 = (ex * ex + ey * ey) + ez * ez;
                    cand[m].i = i;
                    ++m;
                }
            }
    int64_t cap = S->P.max_pts_group;
    if (m > cap) {
        qsort(cand, (size_t)m, sizeof(didx), cmp_didx);
        m = cap;
    }
    int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (m + 1));
    for (int64_t t = 0; t < m; ++t) ids[t] = cand[t].i;
    /* ascending point index */
    for (int64_t t = 1; t < m; ++t) {
        int64_t v = ids[t], s = t - 1;
        while (s >= 0 && ids[s] > v) { ids[s + 1] = ids[s]; --s; }
        ids[s + 1] = v;
    }
    if (out_idx) memcpy(out_idx, ids, sizeof(int64_t) * m);
    free(ids);
    free(cand);
    return m;
}

/* shared set-up of a query batch: query -> instance id, instance list */
typedef struct {
    int64_t nq;
    int64_t* q_inst;     /* -1: bad input (3) or no support (1) */
    uint8_t* q_status0;
    int64_t ni;
    uint64_t* ikey;      /* centre leaf key per instance (sorted) */
    int64_t* ioff;       /* [ni + 1] offsets into iidx */
    int64_t* iidx;       /* point indices per instance */
} qplan;

static void qplan_free(qplan* Q) {
    free(Q->q_inst); free(Q->q_status0); free(Q->ikey); free(Q->ioff); free(Q->iidx);
}

static void qplan_build(const or_surface* S, const float* q, int64_t n, qplan* Q) {
    memset(Q, 0, sizeof(*Q));
    Q->nq = n;
    Q->q_inst = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    Q->q_status0 = (uint8_t*)malloc(n + 1);
    uint64_t* qleaf = (uint64_t*)malloc(sizeof(uint64_t) * (n + 1));
    kidx* R = (kidx*)malloc(sizeof(kidx) * (n + 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {(double)q[3 * i], (double)q[3 * i + 1], (double)q[3 * i + 2]};
        int64_t ijk[3], leaf[3];
        int32_t bit;
        Q->q_inst[i] = -1;
        if (!voxel_ijk(p, S->P.voxel_size, ijk)) { Q->q_status0[i] = ST_BAD_INPUT; qleaf[i] = 0; continue; }
        leaf_of(ijk, leaf, &bit);
        qleaf[i] = pack_key(leaf[0], leaf[1], leaf[2]);
        Q->q_status0[i] = ST_OK;
        R[m].k = qleaf[i]; R[m].i = i; ++m;
    }
    qsort(R, (size_t)m, sizeof(kidx), cmp_kidx);
    /* unique query leaves -> centre leaf */
    int64_t ng = 0;
    for (int64_t i = 0; i < m; ++i) if (i == 0 || R[i].k != R[i - 1].k) ++ng;
    uint64_t* gkey = (uint64_t*)malloc(sizeof(uint64_t) * (ng + 1));
    uint64_t* gcen = (uint64_t*)malloc(sizeof(uint64_t) * (ng + 1));
    uint8_t* gok = (uint8_t*)malloc(ng + 1);
    ng = 0;
    for (int64_t i = 0; i < m; ++i) if (i == 0 || R[i].k != R[i - 1].k) gkey[ng++] = R[i].k;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < ng; ++g) {
        int64_t M[3], C[3];
        unpack_key(gkey[g], M);
        gok[g] = (uint8_t)centre_leaf(S, M, C);
        gcen[g] = gok[g] ? pack_key(C[0], C[1], C[2]) : 0;
    }
    /* unique centres -> instances */
    uint64_t* ck = (uint64_t*)malloc(sizeof(uint64_t) * (ng + 1));
    int64_t nc = 0;
    for (int64_t g = 0; g < ng; ++g) if (gok[g]) ck[nc++] = gcen[g];
    qsort(ck, (size_t)nc, sizeof(uint64_t), cmp_u64);
    int64_t ni = 0;
    for (int64_t i = 0; i < nc; ++i) if (ni == 0 || ck[i] != ck[ni - 1]) ck[ni++] = ck[i];
    Q->ni = ni;
    Q->ikey = ck;
    Q->ioff = (int64_t*)malloc(sizeof(int64_t) * (ni + 1));
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (ni + 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t I = 0; I < ni; ++I) cnt[I] = or_surface_instance(S, ck[I], NULL);
    Q->ioff[0] = 0;
    for (int64_t I = 0; I < ni; ++I) Q->ioff[I + 1] = Q->ioff[I] + cnt[I];
    Q->iidx = (int64_t*)malloc(sizeof(int64_t) * (Q->ioff[ni] + 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t I = 0; I < ni; ++I) or_surface_instance(S, ck[I], Q->iidx + Q->ioff[I]);
    free(cnt);
    /* query -> instance */
    for (int64_t i = 0; i < n; ++i) {
        if (Q->q_status0[i] != ST_OK) continue;
        int64_t g = find_key(gkey, ng, qleaf[i]);
        if (!gok[g]) { Q->q_status0[i] = ST_NO_SUPPORT; continue; }
        Q->q_inst[i] = find_key(Q->ikey, ni, gcen[g]);
    }
    free(gkey); free(gcen); free(gok); free(R); free(qleaf);
}

/* per-instance fitted state */
typedef struct {
    int N;
    double* X;
    double* L;
    double* alpha;
    int ok;
} ifit;

static void ifit_make(const or_surface* S, const qplan* Q, int64_t I, ifit* f) {
    f->N = (int)(Q->ioff[I + 1] - Q->ioff[I]);
    f->X = (double*)malloc(sizeof(double) * 3 * (f->N + 1));
    for (int j = 0; j < f->N; ++j)
        for (int a = 0; a < 3; ++a) f->X[3 * j + a] = S->pts[3 * Q->iidx[Q->ioff[I] + j] + a];
    f->L = (double*)malloc(sizeof(double) * ((int64_t)f->N * (f->N + 1) / 2 + 1));
    f->alpha = (double*)malloc(sizeof(double) * (f->N + 1));
    f->ok = or_gp_fit(f->X, f->N, &S->P, f->L, f->alpha);
}

static void ifit_free(ifit* f) { free(f->X); free(f->L); free(f->alpha); }

int or_query(const or_surface* S, const float* q, int64_t n, int want_var, double* d, double* grad,
             double* var, uint8_t* status, uint64_t* inst_key, int32_t* inst_n) {
    qplan Q;
    qplan_build(S, q, n, &Q);
    /* queries grouped by instance */
    int64_t* qo = (int64_t*)calloc((size_t)(Q.ni + 1), sizeof(int64_t));
    int64_t* ql = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    for (int64_t i = 0; i < n; ++i) if (Q.q_inst[i] >= 0) qo[Q.q_inst[i] + 1]++;
    for (int64_t I = 0; I < Q.ni; ++I) qo[I + 1] += qo[I];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (Q.ni + 1));
        memcpy(fill, qo, sizeof(int64_t) * (Q.ni + 1));
        for (int64_t i = 0; i < n; ++i) if (Q.q_inst[i] >= 0) ql[fill[Q.q_inst[i]]++] = i;
        free(fill);
    }
    for (int64_t i = 0; i < n; ++i) {
        if (Q.q_inst[i] >= 0) continue;
        or_eval r;
        eval_invalid(&r, Q.q_status0[i]);
        if (d) d[i] = r.d;
        if (grad) for (int a = 0; a < 3; ++a) grad[3 * i + a] = 0.0;
        if (var) var[i] = r.v;
        if (status) status[i] = (uint8_t)r.status;
        if (inst_key) inst_key[i] = 0;
        if (inst_n) inst_n[i] = 0;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t I = 0; I < Q.ni; ++I) {
        ifit f;
        ifit_make(S, &Q, I, &f);
        double* kb = (double*)malloc(sizeof(double) * (f.N + 1));
        double* vb = (double*)malloc(sizeof(double) * (f.N + 1));
        for (int64_t t = qo[I]; t < qo[I + 1]; ++t) {
            int64_t i = ql[t];
            double xs[3] = {(double)q[3 * i], (double)q[3 * i + 1], (double)q[3 * i + 2]};
            or_eval r;
            if (!f.ok) eval_invalid(&r, ST_FACTOR_FAIL);
            else gp_eval(f.X, f.N, f.L, f.alpha, xs, &S->P, want_var, kb, vb, &r);
            if (d) d[i] = r.d;
            if (grad) for (int a = 0; a < 3; ++a) grad[3 * i + a] = r.gd[a];
            if (var) var[i] = r.v;
            if (status) status[i] = (uint8_t)r.status;
            if (inst_key) inst_key[i] = Q.ikey[I];
            if (inst_n) inst_n[i] = f.N;
        }
        free(kb); free(vb);
        ifit_free(&f);
    }
    free(qo); free(ql);
    qplan_free(&Q);
    return 0;
}

/*
 * Backward pass of L = sum_q f(d_q) given dL/dd_q (derived from Eq. 1 and Eq. 3):
 *   dL/dx*_q = dL/dd_q * grad d_q;
 *   with obar_q = dL/dd_q * dd/do_q = dL/dd_q * (-l^2 / (o_q d_q)), per instance
 *   abar = sum_q obar_q k_q, lambda = A^-1 abar, and for training point j
 *   dL/dx_j = sum_q obar_q alpha_j k_qj (x*_q - x_j) / l^2
 *             - sum_i (lambda_i alpha_j + lambda_j alpha_i) k_ij (x_i - x_j) / l^2.
 * The contributions of every instance that holds point j are summed into dL/dX[j]
 * in instance order.  Clamped or invalid results contribute zero.
 */
int or_query_backward(const or_surface* S, const float* q, int64_t n, const double* dL_dd,
                      double* dL_dq, double* dL_dX) {
    qplan Q;
    qplan_build(S, q, n, &Q);
    int64_t* qo = (int64_t*)calloc((size_t)(Q.ni + 1), sizeof(int64_t));
    int64_t* ql = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    for (int64_t i = 0; i < n; ++i) if (Q.q_inst[i] >= 0) qo[Q.q_inst[i] + 1]++;
    for (int64_t I = 0; I < Q.ni; ++I) qo[I + 1] += qo[I];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (Q.ni + 1));
        memcpy(fill, qo, sizeof(int64_t) * (Q.ni + 1));
        for (int64_t i = 0; i < n; ++i) if (Q.q_inst[i] >= 0) ql[fill[Q.q_inst[i]]++] = i;
        free(fill);
    }
    if (dL_dq) for (int64_t i = 0; i < 3 * n; ++i) dL_dq[i] = 0.0;
    double* contrib = (double*)calloc((size_t)(3 * Q.ioff[Q.ni] + 1), sizeof(double));
    double l = S->P.lengthscale, l2 = l * l;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t I = 0; I < Q.ni; ++I) {
        ifit f;
        ifit_make(S, &Q, I, &f);
        int N = f.N;
        double* kb = (double*)malloc(sizeof(double) * (N + 1));
        double* abar = (double*)calloc((size_t)(N + 1), sizeof(double));
        double* lam = (double*)malloc(sizeof(double) * (N + 1));
        double* z = (double*)malloc(sizeof(double) * (N + 1));
        double* g = contrib + 3 * Q.ioff[I];
        if (f.ok) {
            for (int64_t t = qo[I]; t < qo[I + 1]; ++t) {
                int64_t i = ql[t];
                double xs[3] = {(double)q[3 * i], (double)q[3 * i + 1], (double)q[3 * i + 2]};
                or_eval r;
                gp_eval(f.X, N, f.L, f.alpha, xs, &S->P, 0, kb, NULL, &r);
                if (dL_dq) for (int a = 0; a < 3; ++a) dL_dq[3 * i + a] = dL_dd[i] * r.gd[a];
                int smooth = r.status == ST_OK && r.d > 0.0 && r.o < 1.0;
                if (!smooth) continue;
                double obar = dL_dd[i] * (-l2 / (r.o * r.d));
                for (int j = 0; j < N; ++j) {
                    abar[j] += obar * kb[j];
                    for (int a = 0; a < 3; ++a)
                        g[3 * j + a] += obar * f.alpha[j] * kb[j] * (xs[a] - f.X[3 * j + a]) / l2;
                }
            }
            forward_subst(f.L, N, abar, z);
            back_subst(f.L, N, z, lam);
            for (int j = 0; j < N; ++j)
                for (int i2 = 0; i2 < N; ++i2) {
                    if (i2 == j) continue;
                    double kij = se_kernel(f.X + 3 * i2, f.X + 3 * j, l);
                    double c = (lam[i2] * f.alpha[j] + lam[j] * f.alpha[i2]) * kij;
                    for (int a = 0; a < 3; ++a) g[3 * j + a] -= c * (f.X[3 * i2 + a] - f.X[3 * j + a]) / l2;
                }
        }
        free(kb); free(abar); free(lam); free(z);
        ifit_free(&f);
    }
    if (dL_dX) {
        for (int64_t i = 0; i < 3 * S->n_pts; ++i) dL_dX[i] = 0.0;
        for (int64_t I = 0; I < Q.ni; ++I)
            for (int64_t t = Q.ioff[I]; t < Q.ioff[I + 1]; ++t)
                for (int a = 0; a < 3; ++a) dL_dX[3 * Q.iidx[t] + a] += contrib[3 * t + a];
    }
    free(contrib); free(qo); free(ql);
    qplan_free(&Q);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* G-GPDF as blended per-leaf GPs (Sec. IV-D, Eq. 10)                                   */
/* ------------------------------------------------------------------------------------ */
/*
 * Each occupied surface leaf is one GP node, trained on the leaf's points (at most
 * max_pts_leaf, the ones nearest to the leaf centre, ties to the lower index).  A query uses
 * the Q nodes nearest to it (FP64 squared distance from the query to the leaf centre, ties
 * to the smaller key) among the occupied leaves in the 27-leaf neighbourhood of the query
 * leaf's centre leaf (the same centre rule as the neighbourhood GP).  Eq. 10 is read as a
 * smooth minimum: d = sum_q d_q w_q / sum_q w_q with w_q = exp(-lambda (d_q - min d)), over the
 * nodes whose result is valid; the gradient is the plain average of the valid nodes'
 * gradients ("directly average"), the variance the same weighted average as d.
 */
static int64_t leaf_points_capped(const or_surface* S, int64_t l, int cap, int64_t* out) {
    int64_t n = S->off[l + 1] - S->off[l];
    int64_t L[3];
    unpack_key(S->lkey[l], L);
    double vs = S->P.voxel_size, c[3];
    for (int a = 0; a < 3; ++a) c[a] = ((double)(8 * L[a]) + 3.5) * vs;
    didx* cand = (didx*)malloc(sizeof(didx) * (n + 1));
    for (int64_t t = 0; t < n; ++t) {
        int64_t i = S->idx[S->off[l] + t];
        const double* x = S->pts + 3 * i;
        double ex = x[0] - c[0], ey = x[1] - c[1], ez = x[2] - c[2];
        cand[t].d2 = (ex * ex + ey * ey) + ez * ez;
        cand[t].i = i;
    }
    int64_t m = n;
    if (m > cap) {
        qsort(cand, (size_t)m, sizeof(didx), cmp_didx);
        m = cap;
    }
    for (int64_t t = 0; t < m; ++t) out[t] = cand[t].i;
    for (int64_t t = 1; t < m; ++t) {
        int64_t v = out[t], u = t - 1;
        while (u >= 0 && out[u] > v) { out[u + 1] = out[u]; --u; }
        out[u + 1] = v;
    }
    free(cand);
    return m;
}

typedef struct {
    double d2;
    uint64_t key;
    int64_t l;
} node_c;

static int cmp_node(const void* a, const void* b) {
    const node_c* x = (const node_c*)a;
    const node_c* y = (const node_c*)b;
    if (x->d2 != y->d2) return x->d2 < y->d2 ? -1 : 1;
    return (x->key > y->key) - (x->key < y->key);
}

/* The nodes of query point xs whose centre leaf is C: the occupied leaves of C's 27-leaf
 * neighbourhood, nearest first (FP64 squared distance to the leaf centre, ties to the
 * smaller key), at most Qmax of them, in nc[0 .. return value). */
static int smooth_select(const or_surface* S, const double xs[3], const int64_t C[3], int Qmax, node_c nc[27]) {
    int nn = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t F[3] = {C[0] + dx, C[1] + dy, C[2] + dz};
                uint64_t k = pack_key(F[0], F[1], F[2]);
                int64_t l = find_key(S->lkey, S->nl, k);
                if (l < 0) continue;
                double e2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double c = ((double)(8 * F[a]) + 3.5) * S->P.voxel_size;
                    double e = xs[a] - c;
                    e2 += e * e;
                }
                nc[nn].d2 = e2; nc[nn].key = k; nc[nn].l = l; ++nn;
            }
    qsort(nc, (size_t)nn, sizeof(node_c), cmp_node);
    return nn > Qmax ? Qmax : nn;
}

/* Node choice of or_query_smooth for each query: keys[i * Qmax + t] = leaf key of its node of
 * rank t, 0 past the last node (and for queries without a centre leaf). */
int or_query_smooth_nodes(const or_surface* S, const float* q, int64_t n, int Qmax, uint64_t* keys) {
    for (int64_t i = 0; i < n; ++i) {
        for (int t = 0; t < Qmax; ++t) keys[i * Qmax + t] = 0;
        double p[3] = {(double)q[3 * i], (double)q[3 * i + 1], (double)q[3 * i + 2]};
        int64_t ijk[3], M[3], C[3];
        int32_t bit;
        if (!voxel_ijk(p, S->P.voxel_size, ijk)) continue;
        leaf_of(ijk, M, &bit);
        if (!centre_leaf(S, M, C)) continue;
        node_c nc[27];
        int nn = smooth_select(S, p, C, Qmax, nc);
        for (int t = 0; t < nn; ++t) keys[i * Qmax + t] = nc[t].key;
    }
    return 0;
}

/* Training points of the node GP of leaf `key` (the leaf's points, at most cap of them, those
 * nearest the leaf centre), as sorted point indices in out (may be NULL); returns their count,
 * 0 for an unoccupied leaf. */
int64_t or_surface_leaf_capped(const or_surface* S, uint64_t key, int cap, int64_t* out) {
    int64_t l = find_key(S->lkey, S->nl, key);
    if (l < 0) return 0;
    int64_t n = S->off[l + 1] - S->off[l];
    int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    int64_t m = leaf_points_capped(S, l, cap, tmp);
    if (out) memcpy(out, tmp, sizeof(int64_t) * m);
    free(tmp);
    return m;
}

int or_query_smooth(const or_surface* S, const float* q, int64_t n, int Qmax, double lambda, int want_var,
                    double* d, double* grad, double* var, uint8_t* status, int32_t* n_nodes) {
    const or_params* P = &S->P;
    /* fit every occupied leaf lazily, once (cache by leaf index) */
    ifit* fits = (ifit*)calloc((size_t)(S->nl + 1), sizeof(ifit));
    uint8_t* have = (uint8_t*)calloc((size_t)(S->nl + 1), 1);
    int cap = P->max_pts_leaf;
    /* which leaves are needed: first pass, serial (cheap) */
    int64_t* need_list = (int64_t*)malloc(sizeof(int64_t) * (S->nl + 1));
    int64_t n_need = 0;
    int64_t* q_c = (int64_t*)malloc(sizeof(int64_t) * 3 * (n + 1));
    uint8_t* q_ok = (uint8_t*)malloc(n + 1);
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {(double)q[3 * i], (double)q[3 * i + 1], (double)q[3 * i + 2]};
        int64_t ijk[3], M[3], C[3];
        int32_t bit;
        q_ok[i] = 0;
        if (!voxel_ijk(p, P->voxel_size, ijk)) continue;
        leaf_of(ijk, M, &bit);
        if (!centre_leaf(S, M, C)) { q_ok[i] = 2; continue; }
        q_ok[i] = 1;
        for (int a = 0; a < 3; ++a) q_c[3 * i + a] = C[a];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t l = find_key(S->lkey, S->nl, pack_key(C[0] + dx, C[1] + dy, C[2] + dz));
                    if (l >= 0 && !have[l]) { have[l] = 1; need_list[n_need++] = l; }
                }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < n_need; ++t) {
        int64_t l = need_list[t];
        int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (S->off[l + 1] - S->off[l] + 1));
        int64_t m = leaf_points_capped(S, l, cap, ids);
        ifit* f = &fits[l];
        f->N = (int)m;
        f->X = (double*)malloc(sizeof(double) * 3 * (m + 1));
        for (int64_t j = 0; j < m; ++j)
            for (int a = 0; a < 3; ++a) f->X[3 * j + a] = S->pts[3 * ids[j] + a];
        f->L = (double*)malloc(sizeof(double) * ((int64_t)m * (m + 1) / 2 + 1));
        f->alpha = (double*)malloc(sizeof(double) * (m + 1));
        f->ok = or_gp_fit(f->X, f->N, P, f->L, f->alpha);
        free(ids);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        or_eval r0;
        if (q_ok[i] != 1) {
            eval_invalid(&r0, q_ok[i] == 0 ? ST_BAD_INPUT : ST_NO_SUPPORT);
            if (d) d[i] = r0.d;
            if (grad) for (int a = 0; a < 3; ++a) grad[3 * i + a] = 0.0;
            if (var) var[i] = r0.v;
            if (status) status[i] = (uint8_t)r0.status;
            if (n_nodes) n_nodes[i] = 0;
            continue;
        }
        double xs[3] = {(double)q[3 * i], (double)q[3 * i + 1], (double)q[3 * i + 2]};
        node_c nc[27];
        int nn = smooth_select(S, xs, q_c + 3 * i, Qmax, nc);
        double dq[27], vq[27], gq[27][3];
        int stq[27];
        int n_ok = 0, first_status = ST_NO_SUPPORT;
        double dmin = INFINITY;
        for (int t = 0; t < nn; ++t) {
            ifit* f = &fits[nc[t].l];
            or_eval r;
            double* kb = (double*)malloc(sizeof(double) * (f->N + 1));
            double* vb = (double*)malloc(sizeof(double) * (f->N + 1));
            if (!f->ok) eval_invalid(&r, ST_FACTOR_FAIL);
            else gp_eval(f->X, f->N, f->L, f->alpha, xs, P, want_var, kb, vb, &r);
            free(kb); free(vb);
            dq[t] = r.d; vq[t] = r.v; stq[t] = r.status;
            for (int a = 0; a < 3; ++a) gq[t][a] = r.gd[a];
            if (t == 0) first_status = r.status;
            if (r.status == ST_OK) { ++n_ok; if (r.d < dmin) dmin = r.d; }
        }
        double dd, g[3] = {0.0, 0.0, 0.0}, vv = NAN;
        int st;
        if (n_ok == 0) {
            st = first_status;
            dd = (st == ST_CLAMPED) ? P->d_max : INFINITY;
            vv = INFINITY;
        } else {
            double sw = 0.0, swd = 0.0, swv = 0.0;
            for (int t = 0; t < nn; ++t) {
                if (stq[t] != ST_OK) continue;
                double w = exp(-lambda * (dq[t] - dmin));
                sw += w; swd += w * dq[t]; swv += w * vq[t];
                for (int a = 0; a < 3; ++a) g[a] += gq[t][a];
            }
            dd = swd / sw;
            vv = swv / sw;
            for (int a = 0; a < 3; ++a) g[a] /= (double)n_ok;
            st = ST_OK;
        }
        if (d) d[i] = dd;
        if (grad) for (int a = 0; a < 3; ++a) grad[3 * i + a] = g[a];
        if (var) var[i] = want_var ? vv : NAN;
        if (status) status[i] = (uint8_t)st;
        if (n_nodes) n_nodes[i] = nn;
    }
    for (int64_t l = 0; l < S->nl; ++l) if (have[l]) ifit_free(&fits[l]);
    free(fits); free(have); free(need_list); free(q_c); free(q_ok);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
