/*
 * Oracle-S: the exact FP64 normal equations of one bundle-adjustment window, stored as a
 * block-sparse matrix and solved with a generic block-sparse Cholesky factorisation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU legs
 * may load this library (through oracle/ba_sparse.py).  It shares no code with the CUDA
 * library and includes none of its headers.
 *
 * What it computes (cuVSLAM, arXiv 2506.04359, Sec. 2.2 "3D module"): for the
 * reprojection residual r_n = pi(T^cb_k T^bw_i p^w_j) - o_{j,k} (Eq. r^repr) and the
 * objective 1/2 sum rho(|r_n|^2) (Eq. argmin, Sigma = I, Huber kernel), the damped
 * Gauss-Newton system (H + lambda D) delta = -g with H = sum w J^T J, g = sum w J^T r over
 * all free keyframe twists and landmark coordinates: the same system the dense oracle
 * (oracle/ba.py) forms and factors with LAPACK.  Here the system is never dense:
 *
 *   1. per observation: residual, validity (camera depth > z_min), Huber weight and the
 *      2x6 / 2x3 Jacobians, exactly as the dense oracle's `residuals` and `jacobians`;
 *   2. H is accumulated into its nonzero blocks only (3x3 landmark, 6x6 keyframe, 6x3
 *      keyframe-landmark) and g into a vector;
 *   3. D = diag(H) floored at 1e-12 max(diag H); A = H + lambda D;
 *   4. A = L L^T by a generic block-sparse Cholesky: block columns ordered landmarks first,
 *      then free keyframes; a symbolic analysis derives the factor's block pattern from A's
 *      by the elimination-tree rule (the pattern of column c is A's pattern below c merged
 *      with the patterns of c's children minus c); the numeric factorisation is
 *      right-looking (factor the diagonal block of column c, solve the blocks below it,
 *      subtract their outer products from the later columns);
 *   5. forward and backward block substitution give delta.
 * The factorisation knows nothing about cameras or landmarks: it sees block columns and a
 * pattern.  (With landmarks first, the elimination of the landmark columns is what the
 * paper calls the Schur complement; this code does not single it out.)
 *
 * Parallelism (OpenMP, optional) never changes a result: per-observation work writes
 * per-observation slots; keyframe sums are accumulated per fixed landmark chunk and added
 * in chunk order; the leading block columns that no earlier column updates are factored
 * concurrently, and their updates are applied target column by target column, each target
 * block receiving them in ascending source-column order, as the sequential right-looking
 * loop would.  Compiled with -ffp-contract=off, so no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BMAX 6          /* largest block size (a keyframe twist) */
#define NCHUNK 256      /* fixed landmark chunks for the keyframe sums */
#define DIAG_FLOOR 1e-12

typedef struct bs_window {
  int K, C, M, N, fixed_kf;
  int nfree, nb;                 /* free keyframes; block columns = M + nfree */
  int64_t n_c, n_f;              /* 6 nfree; n_c + 3 M */
  const double *intr, *T_cb, *uv;
  const int32_t *kf, *cam, *lm;
  double huber, zmin;
  int threads;
  /* observations grouped by landmark, in caller order within a landmark */
  int64_t *lm_obs_off;           /* M + 1 */
  int32_t *lm_obs;               /* N */
  int32_t *kf_block;             /* K: block column of each keyframe, -1 for the fixed one */
  int *bsz;                      /* nb: block size */
  int64_t *xoff;                 /* nb: offset in the solution vector (keyframes first, then
                                    landmarks, as the dense oracle orders its columns) */
  /* pattern of the factor below the diagonal, by block column; rows ascending */
  int64_t *l_cp;                 /* nb + 1 */
  int32_t *l_rows;
  int64_t *l_val;                /* value offset of each off-diagonal block */
  int64_t *d_val;                /* nb: value offset of each diagonal block */
  double *val;
  int64_t n_val;
  int n_indep;                   /* leading columns no earlier column updates */
  /* for target columns >= n_indep: the updating (source column, index in its rows) pairs */
  int64_t *u_cp;
  int32_t *u_src, *u_idx;
  /* per observation: value offset of its (keyframe, landmark) block of H, -1 if fixed */
  int64_t *obs_blk;
  /* work */
  double *rho, *ssq;
  uint8_t *vflag, *iflag;
} bs_window;

/* --------------------------------------------------------------- observation model */

/* X_b = R_i p_j + t_i, X_c = R^cb_k X_b + t^cb_k and r = pi(X_c) - o; 0 if Z_c <= z_min. */
static int residual(const bs_window* w, const double* poses, const double* lms, int64_t n, double Xb[3],
                    double Xc[3], double r[2]) {
  const double* T = poses + 12 * (int64_t)w->kf[n];
  const double* p = lms + 3 * (int64_t)w->lm[n];
  const double* Q = w->T_cb + 12 * (int64_t)w->cam[n];
  const double* f = w->intr + 4 * (int64_t)w->cam[n];
  for (int a = 0; a < 3; ++a) Xb[a] = T[4 * a] * p[0] + T[4 * a + 1] * p[1] + T[4 * a + 2] * p[2] + T[4 * a + 3];
  for (int a = 0; a < 3; ++a) Xc[a] = Q[4 * a] * Xb[0] + Q[4 * a + 1] * Xb[1] + Q[4 * a + 2] * Xb[2] + Q[4 * a + 3];
  if (!(Xc[2] > w->zmin)) {
    r[0] = r[1] = 0.0;
    return 0;
  }
  r[0] = f[0] * Xc[0] / Xc[2] + f[2] - w->uv[2 * n];
  r[1] = f[1] * Xc[1] / Xc[2] + f[3] - w->uv[2 * n + 1];
  return 1;
}

/* J_pose = dpi/dX_c R^cb [I | -[X_b]x] (2x6) and J_lm = dpi/dX_c R^cb R_i (2x3). */
static void jacobians(const bs_window* w, const double* poses, int64_t n, const double Xb[3], const double Xc[3],
                      double Jp[2][6], double Jl[2][3]) {
  const double* T = poses + 12 * (int64_t)w->kf[n];
  const double* Q = w->T_cb + 12 * (int64_t)w->cam[n];
  const double* f = w->intr + 4 * (int64_t)w->cam[n];
  const double Z = Xc[2];
  const double Jpi[2][3] = {{f[0] / Z, 0.0, -f[0] * Xc[0] / (Z * Z)}, {0.0, f[1] / Z, -f[1] * Xc[1] / (Z * Z)}};
  double A[2][3];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b) A[a][b] = Jpi[a][0] * Q[b] + Jpi[a][1] * Q[4 + b] + Jpi[a][2] * Q[8 + b];
  /* -[X_b]x */
  const double S[3][3] = {{0.0, Xb[2], -Xb[1]}, {-Xb[2], 0.0, Xb[0]}, {Xb[1], -Xb[0], 0.0}};
  for (int a = 0; a < 2; ++a) {
    for (int b = 0; b < 3; ++b) {
      Jp[a][b] = A[a][b];
      Jp[a][3 + b] = A[a][0] * S[0][b] + A[a][1] * S[1][b] + A[a][2] * S[2][b];
      Jl[a][b] = A[a][0] * T[b] + A[a][1] * T[4 + b] + A[a][2] * T[8 + b];
    }
  }
}

/* Huber on the squared norm s: rho(s) and the IRLS weight w = drho/ds. */
static void huber(double s, double delta, double* rho, double* wt, int* inlier) {
  const double e = sqrt(s);
  *inlier = e <= delta;
  *rho = *inlier ? s : 2.0 * delta * e - delta * delta;
  *wt = *inlier ? 1.0 : delta / e;
}

/* ---------------------------------------------------------------- small dense blocks */

/* In-place Cholesky of an n x n row-major block (lower triangle used, upper zeroed).
 * Returns 0 if a pivot is not positive or not finite. */
static int chol_block(double* a, int n) {
  for (int j = 0; j < n; ++j) {
    double d = a[j * n + j];
    for (int k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
    if (!(d > 0.0) || !isfinite(d)) return 0;
    const double l = sqrt(d);
    a[j * n + j] = l;
    for (int i = j + 1; i < n; ++i) {
      double s = a[i * n + j];
      for (int k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = s / l;
    }
    for (int i = 0; i < j; ++i) a[i * n + j] = 0.0;
  }
  return 1;
}

/* B (m x n) <- B L^-T with L (n x n) lower triangular: row by row, L x = b. */
static void trsm_right_lt(double* B, int m, const double* L, int n) {
  for (int i = 0; i < m; ++i) {
    double* b = B + i * n;
    for (int j = 0; j < n; ++j) {
      double s = b[j];
      for (int k = 0; k < j; ++k) s -= L[j * n + k] * b[k];
      b[j] = s / L[j * n + j];
    }
  }
}

/* C (m x p) -= A (m x n) B^T (B is p x n). */
static void gemm_sub_nt(double* Cm, const double* A, const double* B, int m, int n, int p) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[j * n + k];
      Cm[i * p + j] -= s;
    }
}

/* ------------------------------------------------------------------ pattern helpers */

static int cmp_i32(const void* a, const void* b) {
  const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* position of row r in the sorted rows of column c, or -1 */
static int64_t find_row(const bs_window* w, int c, int32_t r) {
  int64_t lo = w->l_cp[c], hi = w->l_cp[c + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (w->l_rows[mid] < r)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo < w->l_cp[c + 1] && w->l_rows[lo] == r ? lo : -1;
}

typedef struct {
  int32_t* p;
  int64_t n, cap;
} ivec;

static int ivec_push(ivec* v, int32_t x) {
  if (v->n == v->cap) {
    const int64_t cap = v->cap ? 2 * v->cap : 1024;
    int32_t* q = (int32_t*)realloc(v->p, (size_t)cap * sizeof(int32_t));
    if (!q) return 0;
    v->p = q;
    v->cap = cap;
  }
  v->p[v->n++] = x;
  return 1;
}

void bs_destroy(bs_window* w);
void bs_solve_rhs(const bs_window* w, const double* b, double* x);

/* ------------------------------------------------------------------------ analysis */

/* Analyse a window: group observations, build H's block pattern (landmark columns first,
 * rows = the free keyframes observing the landmark), derive the factor's pattern and the
 * update lists.  Arrays are borrowed and must outlive the handle.  NULL on failure. */
bs_window* bs_create(int K, int C, int M, int N, int fixed_kf, const double* intr, const double* T_cb,
                     const int32_t* kf, const int32_t* cam, const int32_t* lm, const double* uv, int threads) {
  if (K < 2 || C < 1 || M < 1 || N < 1 || fixed_kf < 0 || fixed_kf >= K) return NULL;
  for (int64_t n = 0; n < N; ++n)
    if (kf[n] < 0 || kf[n] >= K || cam[n] < 0 || cam[n] >= C || lm[n] < 0 || lm[n] >= M) return NULL;
  bs_window* w = (bs_window*)calloc(1, sizeof(bs_window));
  if (!w) return NULL;
  w->K = K, w->C = C, w->M = M, w->N = N, w->fixed_kf = fixed_kf;
  w->intr = intr, w->T_cb = T_cb, w->kf = kf, w->cam = cam, w->lm = lm, w->uv = uv;
  w->threads = threads;
  w->nfree = K - 1;
  w->nb = M + w->nfree;
  w->n_c = 6 * (int64_t)w->nfree;
  w->n_f = w->n_c + 3 * (int64_t)M;
  const int nb = w->nb;

  w->kf_block = (int32_t*)malloc(sizeof(int32_t) * K);
  w->bsz = (int*)malloc(sizeof(int) * nb);
  w->xoff = (int64_t*)malloc(sizeof(int64_t) * nb);
  w->lm_obs_off = (int64_t*)calloc((size_t)M + 1, sizeof(int64_t));
  w->lm_obs = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  w->obs_blk = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  w->rho = (double*)malloc(sizeof(double) * (size_t)N);
  w->ssq = (double*)malloc(sizeof(double) * (size_t)N);
  w->vflag = (uint8_t*)malloc((size_t)N);
  w->iflag = (uint8_t*)malloc((size_t)N);
  if (!w->kf_block || !w->bsz || !w->xoff || !w->lm_obs_off || !w->lm_obs || !w->obs_blk || !w->rho || !w->ssq ||
      !w->vflag || !w->iflag) {
    bs_destroy(w);
    return NULL;
  }
  for (int i = 0, b = 0; i < K; ++i) w->kf_block[i] = i == fixed_kf ? -1 : M + b++;
  for (int c = 0; c < nb; ++c) {
    w->bsz[c] = c < M ? 3 : 6;
    w->xoff[c] = c < M ? w->n_c + 3 * (int64_t)c : 6 * (int64_t)(c - M);
  }
  /* counting sort of observations by landmark (stable) */
  for (int64_t n = 0; n < N; ++n) w->lm_obs_off[lm[n] + 1]++;
  for (int j = 0; j < M; ++j) w->lm_obs_off[j + 1] += w->lm_obs_off[j];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    if (!fill) {
      bs_destroy(w);
      return NULL;
    }
    memcpy(fill, w->lm_obs_off, sizeof(int64_t) * (size_t)M);
    for (int64_t n = 0; n < N; ++n) w->lm_obs[fill[lm[n]]++] = (int32_t)n;
    free(fill);
  }

  /* H's pattern below the diagonal: column j (landmark) has the block rows of the free
   * keyframes that observe it; keyframe columns have none (an observation couples one
   * keyframe with one landmark). */
  int64_t* a_cp = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
  ivec a_rows = {0};
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * nb);
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * nb);
  if (!a_cp || !mark || !tmp) {
    free(a_cp), free(mark), free(tmp);
    bs_destroy(w);
    return NULL;
  }
  for (int c = 0; c < nb; ++c) mark[c] = -1;
  for (int c = 0; c < nb; ++c) {
    int nt = 0;
    if (c < M)
      for (int64_t q = w->lm_obs_off[c]; q < w->lm_obs_off[c + 1]; ++q) {
        const int32_t r = w->kf_block[kf[w->lm_obs[q]]];
        if (r > c && mark[r] != c) mark[r] = c, tmp[nt++] = r;
      }
    qsort(tmp, nt, sizeof(int32_t), cmp_i32);
    for (int k = 0; k < nt; ++k) ivec_push(&a_rows, tmp[k]);
    a_cp[c + 1] = a_rows.n;
  }

  /* symbolic factorisation: pattern(c) = A's rows below c, merged with the patterns of the
   * children of c (columns whose first row is c), minus c itself */
  int32_t* child_head = (int32_t*)malloc(sizeof(int32_t) * nb);
  int32_t* child_next = (int32_t*)malloc(sizeof(int32_t) * nb);
  w->l_cp = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
  ivec l_rows = {0};
  if (!child_head || !child_next || !w->l_cp) {
    free(a_cp), free(mark), free(tmp), free(a_rows.p), free(child_head), free(child_next);
    bs_destroy(w);
    return NULL;
  }
  for (int c = 0; c < nb; ++c) child_head[c] = -1, mark[c] = -1;
  for (int c = 0; c < nb; ++c) {
    int nt = 0;
    for (int64_t q = a_cp[c]; q < a_cp[c + 1]; ++q) {
      const int32_t r = a_rows.p[q];
      if (mark[r] != c) mark[r] = c, tmp[nt++] = r;
    }
    for (int32_t k = child_head[c]; k >= 0; k = child_next[k])
      for (int64_t q = w->l_cp[k]; q < w->l_cp[k + 1]; ++q) {
        const int32_t r = l_rows.p[q];
        if (r != c && mark[r] != c) mark[r] = c, tmp[nt++] = r;
      }
    qsort(tmp, nt, sizeof(int32_t), cmp_i32);
    for (int k = 0; k < nt; ++k) ivec_push(&l_rows, tmp[k]);
    w->l_cp[c + 1] = l_rows.n;
    if (nt > 0) child_next[c] = child_head[tmp[0]], child_head[tmp[0]] = c;
  }
  w->l_rows = l_rows.p;
  free(a_cp), free(a_rows.p), free(child_head), free(child_next);

  /* value offsets: diagonal blocks, then each column's blocks below the diagonal */
  const int64_t nnz = w->l_cp[nb];
  w->d_val = (int64_t*)malloc(sizeof(int64_t) * nb);
  w->l_val = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  if (!w->d_val || !w->l_val) {
    free(mark), free(tmp);
    bs_destroy(w);
    return NULL;
  }
  int64_t off = 0;
  for (int c = 0; c < nb; ++c) {
    w->d_val[c] = off;
    off += w->bsz[c] * w->bsz[c];
    for (int64_t q = w->l_cp[c]; q < w->l_cp[c + 1]; ++q) {
      w->l_val[q] = off;
      off += w->bsz[w->l_rows[q]] * w->bsz[c];
    }
  }
  w->n_val = off;
  w->val = (double*)malloc(sizeof(double) * (size_t)off);

  /* leading columns that no earlier column updates: they depend on A alone */
  for (int c = 0; c < nb; ++c) mark[c] = 0;
  for (int64_t q = 0; q < nnz; ++q) mark[w->l_rows[q]] = 1;
  w->n_indep = 0;
  while (w->n_indep < nb && !mark[w->n_indep]) w->n_indep++;
  /* their updates, listed by target column in ascending source order */
  w->u_cp = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
  const int64_t n_upd = w->l_cp[w->n_indep];
  w->u_src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_upd > 0 ? n_upd : 1));
  w->u_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_upd > 0 ? n_upd : 1));
  if (!w->val || !w->u_cp || !w->u_src || !w->u_idx) {
    free(mark), free(tmp);
    bs_destroy(w);
    return NULL;
  }
  for (int64_t q = 0; q < n_upd; ++q) w->u_cp[w->l_rows[q] + 1]++;
  for (int c = 0; c < nb; ++c) w->u_cp[c + 1] += w->u_cp[c];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    memcpy(fill, w->u_cp, sizeof(int64_t) * (size_t)nb);
    for (int c = 0; c < w->n_indep; ++c)
      for (int64_t q = w->l_cp[c]; q < w->l_cp[c + 1]; ++q) {
        const int32_t r = w->l_rows[q];
        w->u_src[fill[r]] = c;
        w->u_idx[fill[r]] = (int32_t)(q - w->l_cp[c]);
        fill[r]++;
      }
    free(fill);
  }
  /* each observation's (keyframe, landmark) block of H below the diagonal */
  for (int64_t n = 0; n < N; ++n) {
    const int32_t r = w->kf_block[kf[n]];
    w->obs_blk[n] = r < 0 ? -1 : w->l_val[find_row(w, lm[n], r)];
  }
  free(mark), free(tmp);
  return w;
}

void bs_destroy(bs_window* w) {
  if (!w) return;
  free(w->lm_obs_off), free(w->lm_obs), free(w->kf_block), free(w->bsz), free(w->xoff);
  free(w->l_cp), free(w->l_rows), free(w->l_val), free(w->d_val), free(w->val);
  free(w->u_cp), free(w->u_src), free(w->u_idx), free(w->obs_blk);
  free(w->rho), free(w->ssq), free(w->vflag), free(w->iflag);
  free(w);
}

/* sizes: n_c, n_f, block columns, factor blocks below the diagonal, factor values, leading
 * independent columns */
void bs_info(const bs_window* w, int64_t out[6]) {
  out[0] = w->n_c, out[1] = w->n_f, out[2] = w->nb, out[3] = w->l_cp[w->nb], out[4] = w->n_val,
  out[5] = w->n_indep;
}

static void set_threads(const bs_window* w) {
#ifdef _OPENMP
  if (w->threads > 0) omp_set_num_threads(w->threads);
#else
  (void)w;
#endif
}

/* ---------------------------------------------------------------------- evaluation */

/* ev[4] = F = 1/2 sum rho over valid observations, sum |r|^2 over them, n_valid, n_inlier
 * (e <= delta).  Sums in observation order. */
void bs_evaluate(bs_window* w, const double* poses, const double* lms, double huber_delta, double z_min,
                 double ev[4]) {
  set_threads(w);
  w->huber = huber_delta, w->zmin = z_min;
  const int64_t N = w->N;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    double Xb[3], Xc[3], r[2], rho, wt;
    int inl = 0;
    const int ok = residual(w, poses, lms, n, Xb, Xc, r);
    const double s = r[0] * r[0] + r[1] * r[1];
    huber(s, huber_delta, &rho, &wt, &inl);
    w->rho[n] = ok ? rho : 0.0;
    w->ssq[n] = ok ? s : 0.0;
    w->vflag[n] = (uint8_t)ok;
    w->iflag[n] = (uint8_t)(ok && inl);
  }
  double F = 0.0, S = 0.0;
  int64_t nv = 0, ni = 0;
  for (int64_t n = 0; n < N; ++n) {
    F += w->rho[n];
    S += w->ssq[n];
    nv += w->vflag[n];
    ni += w->iflag[n];
  }
  ev[0] = 0.5 * F, ev[1] = S, ev[2] = (double)nv, ev[3] = (double)ni;
}

/* -------------------------------------------------------------- normal equations */

/* Assemble H (blocks into the factor's storage, diagonal blocks into hd) and g (solution
 * ordering) at the given state. */
static void assemble(bs_window* w, const double* poses, const double* lms, double* hd, double* g) {
  const int M = w->M, nf = w->nfree, nb = w->nb;
  memset(w->val, 0, sizeof(double) * (size_t)w->n_val);
  memset(g, 0, sizeof(double) * (size_t)w->n_f);
  double* hpp = (double*)calloc((size_t)NCHUNK * nf * 42, sizeof(double));   /* 36 H_pp + 6 g_p */
#pragma omp parallel for schedule(dynamic, 1)
  for (int ch = 0; ch < NCHUNK; ++ch) {
    const int j0 = (int)((int64_t)M * ch / NCHUNK), j1 = (int)((int64_t)M * (ch + 1) / NCHUNK);
    double* part = hpp + (size_t)ch * nf * 42;
    for (int j = j0; j < j1; ++j) {
      double Hll[9] = {0}, gl[3] = {0};
      for (int64_t q = w->lm_obs_off[j]; q < w->lm_obs_off[j + 1]; ++q) {
        const int64_t n = w->lm_obs[q];
        double Xb[3], Xc[3], r[2], rho, wt, Jp[2][6], Jl[2][3];
        int inl;
        if (!residual(w, poses, lms, n, Xb, Xc, r)) continue;
        huber(r[0] * r[0] + r[1] * r[1], w->huber, &rho, &wt, &inl);
        jacobians(w, poses, n, Xb, Xc, Jp, Jl);
        for (int a = 0; a < 3; ++a) {
          for (int b = 0; b < 3; ++b) Hll[3 * a + b] += wt * (Jl[0][a] * Jl[0][b] + Jl[1][a] * Jl[1][b]);
          gl[a] += wt * (Jl[0][a] * r[0] + Jl[1][a] * r[1]);
        }
        if (w->obs_blk[n] < 0) continue;
        const int pb = w->kf_block[w->kf[n]] - M;
        double* W = w->val + w->obs_blk[n];          /* (keyframe, landmark) block, 6 x 3 */
        double* Hp = part + (size_t)pb * 42;
        for (int a = 0; a < 6; ++a) {
          for (int b = 0; b < 3; ++b) W[3 * a + b] += wt * (Jp[0][a] * Jl[0][b] + Jp[1][a] * Jl[1][b]);
          for (int b = 0; b < 6; ++b) Hp[6 * a + b] += wt * (Jp[0][a] * Jp[0][b] + Jp[1][a] * Jp[1][b]);
          Hp[36 + a] += wt * (Jp[0][a] * r[0] + Jp[1][a] * r[1]);
        }
      }
      memcpy(hd + (size_t)9 * j, Hll, sizeof(Hll));
      for (int a = 0; a < 3; ++a) g[w->xoff[j] + a] = gl[a];
    }
  }
  double* hp = hd + (size_t)9 * M;
  memset(hp, 0, sizeof(double) * (size_t)36 * nf);
  for (int ch = 0; ch < NCHUNK; ++ch)
    for (int b = 0; b < nf; ++b) {
      const double* part = hpp + ((size_t)ch * nf + b) * 42;
      for (int k = 0; k < 36; ++k) hp[(size_t)36 * b + k] += part[k];
      for (int a = 0; a < 6; ++a) g[w->xoff[M + b] + a] += part[36 + a];
    }
  free(hpp);
  (void)nb;
}

/* value of block (r, c), r >= c, of the factor's storage */
static double* block_at(const bs_window* w, int r, int c, int64_t q_hint) {
  if (r == c) return w->val + w->d_val[c];
  const int64_t q = q_hint >= 0 ? q_hint : find_row(w, c, r);
  return w->val + w->l_val[q];
}

/* Column c of the factor from its (updated) values: factor the diagonal block, solve the
 * blocks below it.  0 if not positive definite. */
static int factor_column(const bs_window* w, int c) {
  const int s = w->bsz[c];
  double* Lcc = w->val + w->d_val[c];
  if (!chol_block(Lcc, s)) return 0;
  for (int64_t q = w->l_cp[c]; q < w->l_cp[c + 1]; ++q) trsm_right_lt(w->val + w->l_val[q], w->bsz[w->l_rows[q]], Lcc, s);
  return 1;
}

/* Subtract the outer products of column c's blocks rows k1 >= k2 (indices into its rows)
 * from target column r2 = rows(c)[k2]. */
static void update_target(const bs_window* w, int c, int64_t k2) {
  const int s = w->bsz[c];
  const int64_t q2 = w->l_cp[c] + k2;
  const int r2 = w->l_rows[q2];
  const double* B = w->val + w->l_val[q2];
  int64_t hint = w->l_cp[r2];                     /* rows of c below r2 appear in rows(r2) in order */
  for (int64_t q1 = q2; q1 < w->l_cp[c + 1]; ++q1) {
    const int r1 = w->l_rows[q1];
    double* T;
    if (r1 == r2) {
      T = w->val + w->d_val[r2];
    } else {
      while (w->l_rows[hint] < r1) ++hint;       /* present by the symbolic rule */
      T = block_at(w, r1, r2, hint);
    }
    gemm_sub_nt(T, w->val + w->l_val[q1], B, w->bsz[r1], s, w->bsz[r2]);
  }
}

/* delta solving (H + lambda D) delta = -g, with D = diag(H) floored at 1e-12 max diag(H).
 * Also returns g, D (solution ordering) and the evaluation at x.  Returns 1 if the system
 * is positive definite and delta finite, 0 otherwise (delta undefined). */
int bs_linearise_solve(bs_window* w, const double* poses, const double* lms, double lam, double huber_delta,
                       double z_min, double* delta, double* g, double* D, double ev[4]) {
  set_threads(w);
  w->huber = huber_delta, w->zmin = z_min;
  const int M = w->M, nb = w->nb;
  const int64_t n_f = w->n_f;
  bs_evaluate(w, poses, lms, huber_delta, z_min, ev);
  double* hd = (double*)malloc(sizeof(double) * ((size_t)9 * M + (size_t)36 * w->nfree));
  assemble(w, poses, lms, hd, g);
  /* Marquardt diagonal */
  double dmax = 0.0;
  for (int c = 0; c < nb; ++c) {
    const int s = w->bsz[c];
    const double* h = c < M ? hd + (size_t)9 * c : hd + (size_t)9 * M + (size_t)36 * (c - M);
    for (int a = 0; a < s; ++a) {
      D[w->xoff[c] + a] = h[a * s + a];
      if (h[a * s + a] > dmax) dmax = h[a * s + a];
    }
  }
  const double floor_ = DIAG_FLOOR * dmax;
  for (int64_t i = 0; i < n_f; ++i)
    if (D[i] < floor_) D[i] = floor_;
  /* A = H + lambda D into the diagonal blocks */
  for (int c = 0; c < nb; ++c) {
    const int s = w->bsz[c];
    const double* h = c < M ? hd + (size_t)9 * c : hd + (size_t)9 * M + (size_t)36 * (c - M);
    double* a = w->val + w->d_val[c];
    for (int k = 0; k < s * s; ++k) a[k] = h[k];
    for (int k = 0; k < s; ++k) a[k * s + k] += lam * D[w->xoff[c] + k];
  }
  free(hd);

  /* numeric factorisation */
  int ok = 1;
  const int ni = w->n_indep;
#pragma omp parallel for schedule(dynamic, 64) reduction(&& : ok)
  for (int c = 0; c < ni; ++c) ok = factor_column(w, c) && ok;
  if (!ok) return 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int r2 = ni; r2 < nb; ++r2)
    for (int64_t u = w->u_cp[r2]; u < w->u_cp[r2 + 1]; ++u) update_target(w, w->u_src[u], w->u_idx[u]);
  for (int c = ni; c < nb; ++c) {
    if (!factor_column(w, c)) return 0;
    for (int64_t k2 = 0; k2 < w->l_cp[c + 1] - w->l_cp[c]; ++k2) update_target(w, c, k2);
  }

  /* L y = -g, then L^T delta = y */
  for (int64_t i = 0; i < n_f; ++i) delta[i] = -g[i];
  bs_solve_rhs(w, delta, delta);
  for (int64_t i = 0; i < n_f; ++i)
    if (!isfinite(delta[i])) return 0;
  return 1;
}

/* x = (H + lambda D)^-1 b with the factor left by the last successful bs_linearise_solve
 * (solution ordering). */
void bs_solve_rhs(const bs_window* w, const double* b, double* x) {
  const int nb = w->nb;
  for (int64_t i = 0; i < w->n_f; ++i) x[i] = b[i];
  for (int c = 0; c < nb; ++c) {
    const int s = w->bsz[c];
    const double* Lcc = w->val + w->d_val[c];
    double* y = x + w->xoff[c];
    for (int a = 0; a < s; ++a) {
      double t = y[a];
      for (int k = 0; k < a; ++k) t -= Lcc[a * s + k] * y[k];
      y[a] = t / Lcc[a * s + a];
    }
    for (int64_t q = w->l_cp[c]; q < w->l_cp[c + 1]; ++q) {
      const int r = w->l_rows[q], sr = w->bsz[r];
      const double* B = w->val + w->l_val[q];
      double* yr = x + w->xoff[r];
      for (int a = 0; a < sr; ++a)
        for (int k = 0; k < s; ++k) yr[a] -= B[a * s + k] * y[k];
    }
  }
  for (int c = nb - 1; c >= 0; --c) {
    const int s = w->bsz[c];
    const double* Lcc = w->val + w->d_val[c];
    double* y = x + w->xoff[c];
    for (int64_t q = w->l_cp[c]; q < w->l_cp[c + 1]; ++q) {
      const int r = w->l_rows[q], sr = w->bsz[r];
      const double* B = w->val + w->l_val[q];
      const double* xr = x + w->xoff[r];
      for (int k = 0; k < s; ++k)
        for (int a = 0; a < sr; ++a) y[k] -= B[a * s + k] * xr[a];
    }
    for (int a = s - 1; a >= 0; --a) {
      double t = y[a];
      for (int k = a + 1; k < s; ++k) t -= Lcc[k * s + a] * y[k];
      y[a] = t / Lcc[a * s + a];
    }
  }
}

/* The factor's block pattern below the diagonal: cp[nb + 1] column pointers and rows[cp[nb]]
 * (block-column indices: landmarks 0..M-1, then free keyframes in index order). */
void bs_pattern(const bs_window* w, int64_t* cp, int32_t* rows) {
  memcpy(cp, w->l_cp, sizeof(int64_t) * ((size_t)w->nb + 1));
  memcpy(rows, w->l_rows, sizeof(int32_t) * (size_t)w->l_cp[w->nb]);
}
