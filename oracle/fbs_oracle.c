/*
 * Fast Bilateral Solver -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this file.  The product
 * path (the CUDA library) never calls it, and the two share no code.
 *
 * Everything here is the method written out in the paper's order with plain
 * loops, in FP64 (the paper fixes no precision).  Build with
 *     gcc -O2 -ffp-contract=off -fPIC -shared
 * (no FMA contraction, no fast-math) so results are the same on x86-64 and
 * aarch64.
 *
 * Notation.  N pixels, V vertices, C channels.  Key fields are ordered
 * (x, y, l, u, v) as dimensions d = 0..4; the packed 64-bit key holds them
 * MSB -> LSB as y, x, l, u, v in 12-bit fields, so ascending packed key is
 * row-major order of grid cells, then colour.  Neighbour table nbr[v][2d+0]
 * is the -1 neighbour in dimension d and nbr[v][2d+1] the +1 neighbour,
 * -1 when absent.
 *
 * Readings of points the paper leaves open (each is listed with its
 * justification in the design notes):
 *   - quantisation key_d = floor(p_d / sigma_d + 1/2), p = (col, row, l, u, v),
 *     evaluated in FP64; fields outside [0, 4095] are an error;
 *   - vertices are the distinct keys in ascending packed order;
 *   - the blur is Bbar = sum over the 5 dims of the [1, 2, 1] stencil, so
 *     Bbar = 10 I + N with N the sum over existing +-1 neighbours;
 *   - "while not converged" in the bistochastisation is a fixed sweep count;
 *   - 0/0 guards: y0 = 0 where S c = 0; M^-1 = 0 where diag(A) <= 0;
 *     alpha = 0 if d'q <= 0 or delta = 0; beta = 0 if delta_old = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FBSO_FIELD_MAX 4095
#define FBSO_OK 0
#define FBSO_ERR_ARG 1
#define FBSO_ERR_RANGE 2
#define FBSO_ERR_OOM 3

/* bit position of dimension d = (x, y, l, u, v) in the packed key */
static const int kShift[5] = {36, 48, 24, 12, 0};

/* ---------------------------------------------------------------------- */
/* Quantisation: Eq. (2) measures affinity in (x/sxy, y/sxy, l/sl, u/suv,  */
/* v/suv); the simplified grid assigns each pixel to its nearest vertex.   */
/* ---------------------------------------------------------------------- */
static int quantise(double p, double sigma, uint64_t* out)
{
    double k = floor(p / sigma + 0.5);
    if (!(k >= 0.0 && k <= (double)FBSO_FIELD_MAX)) return FBSO_ERR_RANGE; /* NaN fails too */
    *out = (uint64_t)k;
    return FBSO_OK;
}

int fbso_keys(const float* yuv, int64_t H, int64_t W, double sigma_xy, double sigma_l,
              double sigma_uv, uint64_t* keys)
{
    if (!(sigma_xy > 0.0 && sigma_l > 0.0 && sigma_uv > 0.0) || H <= 0 || W <= 0)
        return FBSO_ERR_ARG;
    int64_t N = H * W;
    for (int64_t row = 0; row < H; ++row) {
        for (int64_t col = 0; col < W; ++col) {
            int64_t i = row * W + col;
            double p[5] = {(double)col, (double)row, (double)yuv[i], (double)yuv[N + i],
                           (double)yuv[2 * N + i]};
            double s[5] = {sigma_xy, sigma_xy, sigma_l, sigma_uv, sigma_uv};
            uint64_t key = 0;
            for (int d = 0; d < 5; ++d) {
                uint64_t f;
                int st = quantise(p[d], s[d], &f);
                if (st) return st;
                key |= f << kShift[d];
            }
            keys[i] = key;
        }
    }
    return FBSO_OK;
}

/* ---------------------------------------------------------------------- */
/* Simplified bilateral grid (Eq. (3), (5)): one vertex per distinct key. */
/* ---------------------------------------------------------------------- */
static int cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

/* index of key in sorted unique vkey[0..V), or -1 */
static int64_t find_key(const uint64_t* vkey, int64_t V, uint64_t key)
{
    int64_t lo = 0, hi = V - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (vkey[mid] == key) return mid;
        if (vkey[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Returns V (>= 0) or -FBSO_ERR_OOM.  vkey and m need room for N entries,
 * nbr for 10 N. */
int64_t fbso_grid(const uint64_t* keys, int64_t N, uint64_t* vkey, uint32_t* vid, uint32_t* m,
                  int32_t* nbr)
{
    uint64_t* sorted = (uint64_t*)malloc((size_t)(N > 0 ? N : 1) * sizeof(uint64_t));
    if (!sorted) return -FBSO_ERR_OOM;
    memcpy(sorted, keys, (size_t)N * sizeof(uint64_t));
    qsort(sorted, (size_t)N, sizeof(uint64_t), cmp_u64);
    int64_t V = 0;
    for (int64_t i = 0; i < N; ++i)
        if (i == 0 || sorted[i] != sorted[i - 1]) vkey[V++] = sorted[i];
    free(sorted);

    /* S: pixel i -> vertex vid[i]; m = S 1 (Alg. 1, first step) */
    for (int64_t v = 0; v < V; ++v) m[v] = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t v = find_key(vkey, V, keys[i]);
        vid[i] = (uint32_t)v;
        m[v] += 1;
    }
    /* +-1 neighbours along each of the 5 dimensions; no wrap at field edges */
    for (int64_t v = 0; v < V; ++v) {
        for (int d = 0; d < 5; ++d) {
            uint64_t f = (vkey[v] >> kShift[d]) & FBSO_FIELD_MAX;
            uint64_t unit = (uint64_t)1 << kShift[d];
            int64_t lo = -1, hi = -1;
            if (f > 0) lo = find_key(vkey, V, vkey[v] - unit);
            if (f < FBSO_FIELD_MAX) hi = find_key(vkey, V, vkey[v] + unit);
            nbr[v * 10 + 2 * d + 0] = (int32_t)lo;
            nbr[v * 10 + 2 * d + 1] = (int32_t)hi;
        }
    }
    return V;
}

/* ---------------------------------------------------------------------- */
/* Bistochastisation (supplement Alg. 1): n <- sqrt(n o m / (Bbar n)),     */
/* as a Jacobi sweep (every vertex updated from the previous n).           */
/* Bbar n at v is accumulated as 10 n_v, then + n_u for k = 0..9 in order. */
/* ---------------------------------------------------------------------- */
int fbso_bistochastize(int64_t V, const uint32_t* m, const int32_t* nbr, int iters, double* n)
{
    double* prev = (double*)malloc((size_t)(V > 0 ? V : 1) * sizeof(double));
    if (!prev) return FBSO_ERR_OOM;
    for (int64_t v = 0; v < V; ++v) n[v] = 1.0;
    for (int it = 0; it < iters; ++it) {
        memcpy(prev, n, (size_t)V * sizeof(double));
        for (int64_t v = 0; v < V; ++v) {
            double bn = 10.0 * prev[v];
            for (int k = 0; k < 10; ++k) {
                int32_t u = nbr[v * 10 + k];
                if (u >= 0) bn = bn + prev[u];
            }
            n[v] = sqrt(prev[v] * (double)m[v] / bn);
        }
    }
    free(prev);
    return FBSO_OK;
}

/* ---------------------------------------------------------------------- */
/* Problem construction (Eq. (6)): b = S (c o t), S c, and diag(A) (Sec. 4) */
/* ---------------------------------------------------------------------- */
static void splat_impl(int64_t N, int64_t V, int C, const uint32_t* vid, const float* t,
                       const double* c, double* b, double* sc)
{
    for (int64_t v = 0; v < V; ++v) sc[v] = 0.0;
    for (int64_t k = 0; k < (int64_t)C * V; ++k) b[k] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t v = vid[i];
        sc[v] += c[i];
        for (int ch = 0; ch < C; ++ch) b[ch * V + v] += c[i] * (double)t[ch * N + i];
    }
}

/* b = S (c o t) per channel and S c, summed in FP64 in pixel order */
int fbso_splat(int64_t N, int64_t V, int C, const uint32_t* vid, const float* t, const float* c,
               double* b, double* sc)
{
    double* cd = (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    if (!cd) return FBSO_ERR_OOM;
    for (int64_t i = 0; i < N; ++i) cd[i] = (double)c[i];
    splat_impl(N, V, C, vid, t, cd, b, sc);
    free(cd);
    return FBSO_OK;
}

static int has_neighbour(const int32_t* nbr, int64_t v)
{
    for (int k = 0; k < 10; ++k)
        if (nbr[v * 10 + k] >= 0) return 1;
    return 0;
}

/* diag(A) = lambda (m - Bbar_diag n^2) + S c with Bbar_diag = 10; the
 * smoothness part is exactly 0 for a vertex without neighbours (its row of
 * lambda (D_m - D_n Bbar D_n) vanishes once n^2 = m / 10).  M^-1 = 1/diag(A),
 * 0 where diag(A) <= 0. */
void fbso_diag(int64_t V, const uint32_t* m, const int32_t* nbr, const double* n,
               const double* sc, double lam, double* a, double* minv)
{
    for (int64_t v = 0; v < V; ++v) {
        double smooth = has_neighbour(nbr, v) ? lam * ((double)m[v] - 10.0 * n[v] * n[v]) : 0.0;
        a[v] = smooth + sc[v];
        minv[v] = a[v] > 0.0 ? 1.0 / a[v] : 0.0;
    }
}

/* A z = diag(A) z - lambda D_n N D_n z  (the off-diagonal part of Bbar is N) */
void fbso_apply_A(int64_t V, const int32_t* nbr, const double* n, const double* a, double lam,
                  const double* z, double* out)
{
    for (int64_t v = 0; v < V; ++v) {
        double s = 0.0;
        for (int k = 0; k < 10; ++k) {
            int32_t u = nbr[v * 10 + k];
            if (u >= 0) s += n[u] * z[u];
        }
        out[v] = a[v] * z[v] - lam * n[v] * s;
    }
}

/* flat initialisation (Eq. (13)): y = S(c o t) / S(c), 0 where S c = 0 */
void fbso_flat_init(int64_t V, const double* b, const double* sc, double* y)
{
    for (int64_t v = 0; v < V; ++v) y[v] = sc[v] > 0.0 ? b[v] / sc[v] : 0.0;
}

static double dot(int64_t V, const double* x, const double* y)
{
    double s = 0.0;
    for (int64_t v = 0; v < V; ++v) s += x[v] * y[v];
    return s;
}

/* Preconditioned conjugate gradients (supplement, Algorithm 2; the
 * Hestenes-Stiefel recurrences with a preconditioner), fixed iteration
 * count, one right-hand side.  The preconditioner is a callback so the
 * Jacobi and the hierarchical solves share one loop.  Per iteration:
 *     q = A p;  alpha = rho / p'q;  y += alpha p;  r -= alpha q;
 *     z = M^-1 r;  rho' = r'z;  beta = rho' / rho;  p = z + beta p.
 * The y, r update, z and r'z are one pass over the vertices (z overwrites
 * q, which is no longer needed); rho is the paper's lambda (renamed: the
 * smoothness weight is lambda).  y holds the initial state on entry. */
typedef void (*precond_fn)(const void* ctx, const double* r, double* z);

struct jacobi_ctx { int64_t V; const double* minv; };

static void jacobi_precond(const void* ctx, const double* r, double* z)
{
    const struct jacobi_ctx* J = (const struct jacobi_ctx*)ctx;
    for (int64_t v = 0; v < J->V; ++v) z[v] = J->minv[v] * r[v];
}

static int pcg_core(int64_t V, const int32_t* nbr, const double* n, const double* a, double lam,
                    precond_fn M, const void* mctx, const double* b, double* y, int iters)
{
    size_t sz = (size_t)(V > 0 ? V : 1) * sizeof(double);
    double* r = (double*)malloc(sz);
    double* p = (double*)malloc(sz);
    double* q = (double*)malloc(sz);
    if (!r || !p || !q) { free(r); free(p); free(q); return FBSO_ERR_OOM; }

    /* r = b - A y, p = M^-1 r, rho = r'p */
    fbso_apply_A(V, nbr, n, a, lam, y, q);
    for (int64_t v = 0; v < V; ++v) r[v] = b[v] - q[v];
    M(mctx, r, p);
    double rho = dot(V, r, p);
    for (int it = 0; it < iters; ++it) {
        fbso_apply_A(V, nbr, n, a, lam, p, q);
        const double pq = dot(V, p, q);
        const double alpha = (pq > 0.0 && rho != 0.0) ? rho / pq : 0.0;
        for (int64_t v = 0; v < V; ++v) {
            y[v] += alpha * p[v];
            r[v] -= alpha * q[v];
        }
        M(mctx, r, q);                               /* q now holds z = M^-1 r */
        const double rho_next = dot(V, r, q);
        const double beta = rho != 0.0 ? rho_next / rho : 0.0;
        for (int64_t v = 0; v < V; ++v) p[v] = q[v] + beta * p[v];
        rho = rho_next;
    }
    free(r); free(p); free(q);
    return FBSO_OK;
}

/* Jacobi PCG: M^-1 = 1 / diag(A) (0 where diag(A) <= 0) */
int fbso_pcg(int64_t V, const int32_t* nbr, const double* n, const double* a,
             const double* minv, double lam, const double* b, double* y, int iters)
{
    struct jacobi_ctx J = {V, minv};
    return pcg_core(V, nbr, n, a, lam, jacobi_precond, &J, b, y, iters);
}

/* slice (Eq. (8)): x = S^T y */
/* Single-reduction form of the same PCG (Chronopoulos and Gear, 1989): the
 * iterates equal those of Alg. 2 in exact arithmetic, but both inner
 * products of an iteration are taken at one point, so a parallel
 * implementation needs one global reduction per iteration instead of two.
 * With u = M^-1 r and w = A u kept alongside r, and the search direction p
 * and s = A p updated by recurrences:
 *   gamma = r^T u (Alg. 2's delta),  mu = w^T u,
 *   beta_i = gamma_i / gamma_(i-1),  alpha_i = gamma_i / (mu_i - beta_i gamma_i / alpha_(i-1)),
 *   p <- u + beta p,  s <- w + beta s,  y <- y + alpha p,  r <- r - alpha s,
 *   u <- M^-1 r,  w <- A u.
 * The denominator mu_i - beta_i gamma_i / alpha_(i-1) is p_i^T A p_i.  Guards
 * matching Alg. 2's: beta = 0 when gamma_(i-1) = 0; the correction term is
 * dropped when beta = 0 or alpha_(i-1) = 0; alpha = 0 when gamma = 0 or the
 * denominator is not positive. */
int fbso_pcg_single(int64_t V, const int32_t* nbr, const double* n, const double* a,
                    const double* minv, double lam, const double* b, double* y, int iters)
{
    size_t sz = (size_t)(V > 0 ? V : 1) * sizeof(double);
    double* r = (double*)malloc(sz);
    double* u = (double*)malloc(sz);
    double* w = (double*)malloc(sz);
    double* p = (double*)malloc(sz);
    double* s = (double*)malloc(sz);
    if (!r || !u || !w || !p || !s) {
        free(r); free(u); free(w); free(p); free(s);
        return FBSO_ERR_OOM;
    }
    fbso_apply_A(V, nbr, n, a, lam, y, w);
    for (int64_t v = 0; v < V; ++v) r[v] = b[v] - w[v];
    for (int64_t v = 0; v < V; ++v) u[v] = minv[v] * r[v];
    fbso_apply_A(V, nbr, n, a, lam, u, w);
    double gamma = dot(V, r, u), mu = dot(V, w, u);
    double gamma_old = 0.0, alpha_old = 0.0;
    for (int i = 0; i < iters; ++i) {
        double beta = 0.0, den = mu;
        if (i > 0) {
            beta = gamma_old != 0.0 ? gamma / gamma_old : 0.0;
            if (beta != 0.0 && alpha_old != 0.0) den = mu - beta * gamma / alpha_old;
        }
        double alpha = (gamma != 0.0 && den > 0.0) ? gamma / den : 0.0;
        for (int64_t v = 0; v < V; ++v) {
            p[v] = (i > 0 ? u[v] + beta * p[v] : u[v]);
            s[v] = (i > 0 ? w[v] + beta * s[v] : w[v]);
            y[v] += alpha * p[v];
            r[v] -= alpha * s[v];
            u[v] = minv[v] * r[v];
        }
        fbso_apply_A(V, nbr, n, a, lam, u, w);
        gamma_old = gamma;
        alpha_old = alpha;
        gamma = dot(V, r, u);
        mu = dot(V, w, u);
    }
    free(r); free(u); free(w); free(p); free(s);
    return FBSO_OK;
}

/* ---------------------------------------------------------------------- */
/* Bilateral-space pyramid (supplement, bilateral-space pyramids) and the  */
/* hierarchical preconditioner and initialisation of Sec. 4.               */
/* ---------------------------------------------------------------------- */
/* Level 0 is the grid itself.  Level k+1 halves every key field of level  */
/* k (reading: integer halving, floor -- it reaches a single vertex, as    */
/* the pyramid's top must), de-duplicates in ascending packed order, and   */
/* maps each level-k vertex to its parent.  Returns the number of levels K */
/* (the last has one vertex), or -FBSO_ERR_OOM / -FBSO_ERR_ARG.  sizes[k]  */
/* receives level k's size; parent receives, level after level, the      */
/* parent index of every vertex of levels 0..K-2 (room for 2 V entries     */
/* suffices: every level is at most as large as the one below).           */
static uint64_t halve_key(uint64_t k)
{
    uint64_t out = 0;
    for (int d = 0; d < 5; ++d) {
        uint64_t f = (k >> kShift[d]) & FBSO_FIELD_MAX;
        out |= (f >> 1) << kShift[d];
    }
    return out;
}

int fbso_pyramid(int64_t V, const uint64_t* vkey, int max_levels, int64_t* sizes,
                 int32_t* parent, int64_t parent_cap)
{
    if (V <= 0 || max_levels < 1) return -FBSO_ERR_ARG;
    uint64_t* cur = (uint64_t*)malloc((size_t)V * sizeof(uint64_t));
    uint64_t* nxt = (uint64_t*)malloc((size_t)V * sizeof(uint64_t));
    if (!cur || !nxt) { free(cur); free(nxt); return -FBSO_ERR_OOM; }
    memcpy(cur, vkey, (size_t)V * sizeof(uint64_t));
    int64_t L = V, off = 0;
    int K = 1;
    sizes[0] = V;
    while (L > 1) {
        if (K >= max_levels) { free(cur); free(nxt); return -FBSO_ERR_ARG; }
        for (int64_t i = 0; i < L; ++i) nxt[i] = halve_key(cur[i]);
        uint64_t* h = (uint64_t*)malloc((size_t)L * sizeof(uint64_t));
        if (!h) { free(cur); free(nxt); return -FBSO_ERR_OOM; }
        memcpy(h, nxt, (size_t)L * sizeof(uint64_t));
        qsort(nxt, (size_t)L, sizeof(uint64_t), cmp_u64);
        int64_t L2 = 0;
        for (int64_t i = 0; i < L; ++i)
            if (i == 0 || nxt[i] != nxt[i - 1]) nxt[L2++] = nxt[i];
        if (parent) {
            if (off + L > parent_cap) { free(h); free(cur); free(nxt); return -FBSO_ERR_ARG; }
            for (int64_t i = 0; i < L; ++i) parent[off + i] = (int32_t)find_key(nxt, L2, h[i]);
        }
        free(h);
        off += L;
        sizes[K++] = L2;
        uint64_t* t = cur; cur = nxt; nxt = t;
        L = L2;
    }
    free(cur); free(nxt);
    return K;
}

/* The pyramid the solves use while the hierarchical preconditioner is on. */
static struct {
    int on;
    int K;
    const int64_t* sizes;
    const int32_t* parent;
    double pa, pb, ia, ib;   /* (alpha, beta) of the preconditioner and of the initialisation */
} g_pyr;

/* The paper uses (alpha, beta) = (2, 5) for the preconditioner and (4, 0)
 * for the initialisation. */
void fbso_set_hierarchical(int on, int K, const int64_t* sizes, const int32_t* parent,
                           double prec_alpha, double prec_beta, double init_alpha,
                           double init_beta)
{
    g_pyr.on = on;
    g_pyr.K = K;
    g_pyr.sizes = sizes;
    g_pyr.parent = parent;
    g_pyr.pa = prec_alpha;
    g_pyr.pb = prec_beta;
    g_pyr.ia = init_alpha;
    g_pyr.ib = init_beta;
}

/* P: level values z[0..K) from bilateral-space y (level 0 = y; level k+1
 * sums its children), into one array of sum(sizes) entries. */
static void pyr_lift(const double* y, double* z)
{
    int64_t off = 0;
    for (int64_t i = 0; i < g_pyr.sizes[0]; ++i) z[i] = y[i];
    for (int k = 0; k + 1 < g_pyr.K; ++k) {
        const int64_t L = g_pyr.sizes[k], up = off + L;
        for (int64_t j = 0; j < g_pyr.sizes[k + 1]; ++j) z[up + j] = 0.0;
        for (int64_t i = 0; i < L; ++i) z[up + g_pyr.parent[off + i]] += z[off + i];
        off = up;
    }
}

/* P^T: y = sum over levels of the level values broadcast down to level 0
 * (top down: each level adds its parent's accumulated value). */
static void pyr_collapse(double* z, double* y)
{
    int64_t offs[64];
    offs[0] = 0;
    for (int k = 1; k < g_pyr.K; ++k) offs[k] = offs[k - 1] + g_pyr.sizes[k - 1];
    for (int k = g_pyr.K - 2; k >= 0; --k)
        for (int64_t i = 0; i < g_pyr.sizes[k]; ++i)
            z[offs[k] + i] += z[offs[k + 1] + g_pyr.parent[offs[k] + i]];
    for (int64_t i = 0; i < g_pyr.sizes[0]; ++i) y[i] = z[i];
}

static int64_t pyr_total(void)
{
    int64_t t = 0;
    for (int k = 0; k < g_pyr.K; ++k) t += g_pyr.sizes[k];
    return t;
}

/* level weight: 1 at level 0, alpha^-(beta + k) above */
static double level_weight(int k, double alpha, double beta)
{
    return k == 0 ? 1.0 : pow(alpha, -(beta + k));
}

/* Per-coefficient scale of M_hier^-1 = P^T(w o P(1) o P(.) / P(diag A))
 * (Sec. 4); 0 where P(diag A) <= 0. */
static int hier_coef(const double* a, double* coef)
{
    const int64_t T = pyr_total(), V = g_pyr.sizes[0];
    double* one = (double*)malloc((size_t)V * sizeof(double));
    double* cnt = (double*)malloc((size_t)T * sizeof(double));
    if (!one || !cnt) { free(one); free(cnt); return FBSO_ERR_OOM; }
    for (int64_t i = 0; i < V; ++i) one[i] = 1.0;
    pyr_lift(one, cnt);
    pyr_lift(a, coef);
    int64_t off = 0;
    for (int k = 0; k < g_pyr.K; ++k) {
        const double w = level_weight(k, g_pyr.pa, g_pyr.pb);
        for (int64_t i = 0; i < g_pyr.sizes[k]; ++i) {
            const double dA = coef[off + i];
            coef[off + i] = dA > 0.0 ? w * cnt[off + i] / dA : 0.0;
        }
        off += g_pyr.sizes[k];
    }
    free(one); free(cnt);
    return FBSO_OK;
}

/* s = M_hier^-1 r */
static void hier_apply(const double* coef, const double* r, double* s, double* work)
{
    const int64_t T = pyr_total();
    pyr_lift(r, work);
    for (int64_t i = 0; i < T; ++i) work[i] *= coef[i];
    pyr_collapse(work, s);
}

/* y = P^T(w o P(b) / P(1)) / P^T(w o P(sc) / P(1)) (the push-pull
 * initialisation of Sec. 4); 0 where the denominator is 0. */
static int hier_init(const double* b, const double* sc, double* y)
{
    const int64_t T = pyr_total(), V = g_pyr.sizes[0];
    double* one = (double*)malloc((size_t)V * sizeof(double));
    double* cnt = (double*)malloc((size_t)T * sizeof(double));
    double* zn = (double*)malloc((size_t)T * sizeof(double));
    double* zd = (double*)malloc((size_t)T * sizeof(double));
    double* den = (double*)malloc((size_t)V * sizeof(double));
    if (!one || !cnt || !zn || !zd || !den) {
        free(one); free(cnt); free(zn); free(zd); free(den);
        return FBSO_ERR_OOM;
    }
    for (int64_t i = 0; i < V; ++i) one[i] = 1.0;
    pyr_lift(one, cnt);
    pyr_lift(b, zn);
    pyr_lift(sc, zd);
    int64_t off = 0;
    for (int k = 0; k < g_pyr.K; ++k) {
        const double w = level_weight(k, g_pyr.ia, g_pyr.ib);
        for (int64_t i = 0; i < g_pyr.sizes[k]; ++i) {
            zn[off + i] *= w / cnt[off + i];
            zd[off + i] *= w / cnt[off + i];
        }
        off += g_pyr.sizes[k];
    }
    pyr_collapse(zn, y);
    pyr_collapse(zd, den);
    for (int64_t i = 0; i < V; ++i) y[i] = den[i] > 0.0 ? y[i] / den[i] : 0.0;
    free(one); free(cnt); free(zn); free(zd); free(den);
    return FBSO_OK;
}

/* PCG with M^-1 = M_hier^-1 (the preconditioner of Sec. 4) */
struct hier_ctx { const double* coef; double* work; };

static void hier_precond_cb(const void* ctx, const double* r, double* z)
{
    const struct hier_ctx* H = (const struct hier_ctx*)ctx;
    hier_apply(H->coef, r, z, H->work);
}

static int pcg_hier(int64_t V, const int32_t* nbr, const double* n, const double* a, double lam,
                    const double* b, double* y, int iters)
{
    const int64_t T = pyr_total();
    double* coef = (double*)malloc((size_t)T * sizeof(double));
    double* work = (double*)malloc((size_t)T * sizeof(double));
    int st = (!coef || !work) ? FBSO_ERR_OOM : hier_coef(a, coef);
    if (!st) {
        struct hier_ctx H = {coef, work};
        st = pcg_core(V, nbr, n, a, lam, hier_precond_cb, &H, b, y, iters);
    }
    free(coef); free(work);
    return st;
}

/* The hierarchical preconditioner applied to r (tests) */
int fbso_hier_precond(const double* a, const double* r, double* s)
{
    if (!g_pyr.on) return FBSO_ERR_ARG;
    const int64_t T = pyr_total();
    double* coef = (double*)malloc((size_t)T * sizeof(double));
    double* work = (double*)malloc((size_t)T * sizeof(double));
    int st = (!coef || !work) ? FBSO_ERR_OOM : hier_coef(a, coef);
    if (!st) hier_apply(coef, r, s, work);
    free(coef); free(work);
    return st;
}

/* The hierarchical initialisation of b with weights sc (tests) */
int fbso_hier_init(const double* b, const double* sc, double* y)
{
    if (!g_pyr.on) return FBSO_ERR_ARG;
    return hier_init(b, sc, y);
}

/* Which form the solves below use: 0 = the two-reduction Jacobi PCG of
 * Algorithm 2 (fbso_pcg),
 * 1 = the single-reduction form (fbso_pcg_single).  Process-wide; the test
 * suite sets it around the calls that need it. */
static int g_pcg_form = 0;

void fbso_set_pcg_form(int form) { g_pcg_form = form; }

static int pcg_run(int64_t V, const int32_t* nbr, const double* n, const double* a,
                   const double* minv, double lam, const double* b, double* y, int iters)
{
    if (g_pyr.on) return pcg_hier(V, nbr, n, a, lam, b, y, iters);
    return g_pcg_form == 1 ? fbso_pcg_single(V, nbr, n, a, minv, lam, b, y, iters)
                           : fbso_pcg(V, nbr, n, a, minv, lam, b, y, iters);
}

/* initial state: the flat initialisation, or the hierarchical one */
static int init_run(int64_t V, const double* b, const double* sc, double* y)
{
    if (g_pyr.on) return hier_init(b, sc, y);
    fbso_flat_init(V, b, sc, y);
    return FBSO_OK;
}

void fbso_slice(int64_t N, int64_t V, int C, const uint32_t* vid, const double* y, double* x)
{
    for (int ch = 0; ch < C; ++ch)
        for (int64_t i = 0; i < N; ++i) x[ch * N + i] = y[ch * V + vid[i]];
}

/* One forward solve of C channels sharing A (Sec. 2, Eq. (8); supplement
 * Sec. 4): b, S c, diag(A), flat init, PCG per channel, slice.
 * Outputs y (C x V) and, if x is non-NULL, x (C x N). */
static int solve_impl(int64_t N, int64_t V, int C, const uint32_t* vid, const uint32_t* m,
                      const int32_t* nbr, const double* n, const float* t, const double* c,
                      double lam, int pcg_iters, double* y, double* x)
{
    size_t sv = (size_t)(V > 0 ? V : 1) * sizeof(double);
    double* b = (double*)malloc(sv * (size_t)(C > 0 ? C : 1));
    double* sc = (double*)malloc(sv);
    double* a = (double*)malloc(sv);
    double* minv = (double*)malloc(sv);
    if (!b || !sc || !a || !minv) { free(b); free(sc); free(a); free(minv); return FBSO_ERR_OOM; }
    splat_impl(N, V, C, vid, t, c, b, sc);
    fbso_diag(V, m, nbr, n, sc, lam, a, minv);
    int st = FBSO_OK;
    for (int ch = 0; ch < C && !st; ++ch) {
        st = init_run(V, b + (int64_t)ch * V, sc, y + (int64_t)ch * V);
        if (!st) st = pcg_run(V, nbr, n, a, minv, lam, b + (int64_t)ch * V, y + (int64_t)ch * V, pcg_iters);
    }
    if (!st && x) fbso_slice(N, V, C, vid, y, x);
    free(b); free(sc); free(a); free(minv);
    return st;
}

int fbso_solve(int64_t N, int64_t V, int C, const uint32_t* vid, const uint32_t* m,
               const int32_t* nbr, const double* n, const float* t, const float* c, double lam,
               int pcg_iters, double* y, double* x)
{
    double* cd = (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    if (!cd) return FBSO_ERR_OOM;
    for (int64_t i = 0; i < N; ++i) cd[i] = (double)c[i];
    int st = solve_impl(N, V, C, vid, m, nbr, n, t, cd, lam, pcg_iters, y, x);
    free(cd);
    return st;
}

/* Robust bilateral solver with the Geman-McClure loss (supplement Alg. 3):
 * c <- c_init; repeat irls_iters times { x <- solve(t, c); e <- x - t;
 * c <- 2 s^2 / (s^2 + e^2)^2 }.  Each solve starts afresh from the flat
 * initialisation of the current c.  Returns the last solve's y and x. */
int fbso_solve_robust(int64_t N, int64_t V, const uint32_t* vid, const uint32_t* m,
                      const int32_t* nbr, const double* n, const float* t, const float* c_init,
                      double lam, double sigma_gm, int irls_iters, int pcg_iters, double* y,
                      double* x)
{
    double* c = (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    if (!c) return FBSO_ERR_OOM;
    for (int64_t i = 0; i < N; ++i) c[i] = (double)c_init[i];
    double s2 = sigma_gm * sigma_gm;
    int st = FBSO_OK;
    for (int it = 0; it < irls_iters && !st; ++it) {
        st = solve_impl(N, V, 1, vid, m, nbr, n, t, c, lam, pcg_iters, y, x);
        if (st) break;
        for (int64_t i = 0; i < N; ++i) {
            double e = x[i] - (double)t[i];
            double den = s2 + e * e;
            c[i] = 2.0 * s2 / (den * den);
        }
    }
    free(c);
    return st;
}

/* Backward pass (Sec. 3): g = S dL/dx; z = A^-1 g by the same PCG with the
 * flat initialisation applied to g; dL/dt = c o S^T z;
 * dL/dc = sum_ch [ S^T(-z o yhat) + (S^T z) o t ]  (c is shared by the
 * channels).  yhat is the forward solution (C x V). */
int fbso_backward(int64_t N, int64_t V, int C, const uint32_t* vid, const uint32_t* m,
                  const int32_t* nbr, const double* n, const float* t, const float* c,
                  double lam, int pcg_iters, const double* yhat, const double* dx,
                  double* dt, double* dc)
{
    size_t sv = (size_t)(V > 0 ? V : 1) * sizeof(double);
    double* g = (double*)malloc(sv * (size_t)(C > 0 ? C : 1));
    double* z = (double*)malloc(sv * (size_t)(C > 0 ? C : 1));
    double* sc = (double*)malloc(sv);
    double* a = (double*)malloc(sv);
    double* minv = (double*)malloc(sv);
    if (!g || !z || !sc || !a || !minv) {
        free(g); free(z); free(sc); free(a); free(minv);
        return FBSO_ERR_OOM;
    }
    for (int64_t v = 0; v < V; ++v) sc[v] = 0.0;
    for (int64_t k = 0; k < (int64_t)C * V; ++k) g[k] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        sc[vid[i]] += (double)c[i];
        for (int ch = 0; ch < C; ++ch) g[ch * V + vid[i]] += dx[ch * N + i];
    }
    fbso_diag(V, m, nbr, n, sc, lam, a, minv);
    int st = FBSO_OK;
    for (int ch = 0; ch < C && !st; ++ch) {
        st = init_run(V, g + (int64_t)ch * V, sc, z + (int64_t)ch * V);
        if (!st)
            st = pcg_run(V, nbr, n, a, minv, lam, g + (int64_t)ch * V, z + (int64_t)ch * V,
                         pcg_iters);
    }
    if (!st) {
        for (int64_t i = 0; i < N; ++i) dc[i] = 0.0;
        for (int ch = 0; ch < C; ++ch) {
            for (int64_t i = 0; i < N; ++i) {
                int64_t v = vid[i];
                double zb = z[ch * V + v];                       /* S^T dL/db */
                double zd = -zb * yhat[ch * V + v];              /* S^T dL/ddiag(A) */
                dt[ch * N + i] = (double)c[i] * zb;
                dc[i] += zd + zb * (double)t[ch * N + i];
            }
        }
    }
    free(g); free(z); free(sc); free(a); free(minv);
    return st;
}

/* ---------------------------------------------------------------------
 * Domain transform post-filter (Sec. 5 runs it on the solver's output to
 * smooth the simplified grid's blocky artefacts; the filter is Gastal and
 * Oliveira 2011's recursive formulation, restated here from its
 * published definition).  For a 3-channel guide I (H x W, planar) the step
 * from a pixel to its left (upper) neighbour has length
 *     d = 1 + (sigma_s / sigma_r) * sum_c |I_c(p) - I_c(p')|
 * in the transformed domain.  Iteration i = 1..N filters every row and
 * then every column with a first-order recursive filter of feedback
 * a_i = exp(-sqrt(2) / sigma_i), sigma_i = sigma_s sqrt(3) 2^(N-i) /
 * sqrt(4^N - 1) (the iterations' variances add up to sigma_s^2): along a
 * line with values J and step lengths d (d[k] between k-1 and k),
 *     forward   J[k] <- (1 - a^d[k]) J[k] + a^d[k] J[k-1],     k = 1 .. L-1
 *     backward  J[k] <- (1 - a^d[k+1]) J[k] + a^d[k+1] J[k+1], k = L-2 .. 0.
 * x (C x H x W) is filtered in place. */
static void dt_line(double* J, const double* d, int64_t L, int64_t stride, double a)
{
    for (int64_t k = 1; k < L; ++k) {
        const double w = pow(a, d[k * stride]);
        J[k * stride] = (1.0 - w) * J[k * stride] + w * J[(k - 1) * stride];
    }
    for (int64_t k = L - 2; k >= 0; --k) {
        const double w = pow(a, d[(k + 1) * stride]);
        J[k * stride] = (1.0 - w) * J[k * stride] + w * J[(k + 1) * stride];
    }
}

int fbso_domain_transform(int64_t H, int64_t W, int C, const float* guide, double sigma_s,
                          double sigma_r, int iters, double* x)
{
    if (H < 1 || W < 1 || C < 1 || !(sigma_s > 0) || !(sigma_r > 0) || iters < 1)
        return FBSO_ERR_ARG;
    const int64_t N = H * W;
    double* dh = (double*)calloc((size_t)N, sizeof(double));   /* step from (y, x-1) to (y, x) */
    double* dv = (double*)calloc((size_t)N, sizeof(double));   /* step from (y-1, x) to (y, x) */
    if (!dh || !dv) { free(dh); free(dv); return FBSO_ERR_OOM; }
    const double r = sigma_s / sigma_r;
    for (int64_t yy = 0; yy < H; ++yy)
        for (int64_t xx = 0; xx < W; ++xx) {
            const int64_t p = yy * W + xx;
            double sh = 0.0, sv = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                const double v = guide[ch * N + p];
                if (xx > 0) sh += fabs(v - (double)guide[ch * N + p - 1]);
                if (yy > 0) sv += fabs(v - (double)guide[ch * N + p - W]);
            }
            dh[p] = 1.0 + r * sh;
            dv[p] = 1.0 + r * sv;
        }
    for (int i = 1; i <= iters; ++i) {
        const double sig_i = sigma_s * sqrt(3.0) * pow(2.0, (double)(iters - i)) /
                             sqrt(pow(4.0, (double)iters) - 1.0);
        const double a = exp(-sqrt(2.0) / sig_i);
        for (int ch = 0; ch < C; ++ch) {
            double* X = x + (int64_t)ch * N;
            for (int64_t yy = 0; yy < H; ++yy) dt_line(X + yy * W, dh + yy * W, W, 1, a);
            for (int64_t xx = 0; xx < W; ++xx) dt_line(X + xx, dv + xx, H, W, a);
        }
    }
    free(dh); free(dv);
    return FBSO_OK;
}
