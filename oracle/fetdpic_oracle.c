/*
 * Plain FP64 CPU oracle of the charge-conserving relativistic FETD-PIC step
 * (Na, Moon, Omelchenko, Teixeira, "Relativistic extension of a
 * charge-conservative finite element solver for time-dependent Maxwell-Vlasov
 * equations", arXiv:1707.04333).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark call this file.  It shares no code, header or
 * table with the CUDA library; both are written from the paper.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no FMA contraction, so every expression rounds exactly as written).
 *
 * Readings of places where the paper is silent or garbled:
 *   - local numbering: local edge m of a counter-clockwise triangle is opposite
 *     local node m and runs node m+1 -> node m+2 (indices mod 3); a global edge
 *     (i,j) has i<j and is oriented i -> j;
 *   - barycentric coordinates are evaluated from the gradient form
 *     lambda_m(r) = grad(lambda_m) . (r - r_{m+1});
 *   - 2-D TE: E in-plane on edges, B_z on faces, u carried as a 3-vector with
 *     u_z = 0 preserved;
 *   - Vay: s = 1/(1+|t|^2) and the bracket acts on u'_V (Sec. II.C(b));
 *   - Higuera-Cary: Boris rotation with gamma from the quartic root
 *     sqrt(0.5*(sigma + sqrt(sigma^2 + 4(|beta|^2 + u*^2)))),
 *     sigma = gamma_B^2 - |beta|^2, u* = u^- . beta / c (Sec. II.C(c));
 *   - the walk over crossed triangles and the specular reflection on PEC
 *     walls are not described in the paper; the rule below is this project's.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_EINVAL -1
#define ORA_EMESH -4
#define ORA_EWALK -5

enum { ORA_BORIS = 0, ORA_BORIS_TAN = 1, ORA_VAY = 2, ORA_HC = 3 };

/* Mesh arrays are owned by the caller (numpy); the oracle only fills them. */
typedef struct {
    int nn, nf, ne;
    const double *xy;   /* [nn][2] */
    int *tri;           /* [nf][3] node ids, counter-clockwise */
    int *edge;          /* [ne][2] i<j, oriented i->j */
    int *tri_edge;      /* [nf][3] global edge of local edge m */
    int *tri_sign;      /* [nf][3] +1 if the global edge runs local node m+1 -> m+2 */
    int *tri_nb;        /* [nf][3] triangle across local edge m, -1 on the boundary */
    int *edge_bnd;      /* [ne] 1 if the edge has one triangle (PEC wall) */
    double *d2A;        /* [nf] twice the signed area */
    double *inv2A;      /* [nf] 1/(2A) */
    double *gx, *gy;    /* [nf][3] grad lambda_m */
    double *nx_, *ny_;  /* [nf][3] node coordinates, copied per triangle */
    /* periodic walls (NULL rep = none): node n is identified with node rep[n]
     * (rep[n] == n for every node that is not an image); an image sits at its
     * representative's position plus (tx, ty).  tri_shift[3f+m] in {-1,0,1}:
     * crossing local edge m of triangle f translates the position by
     * tri_shift * (tx, ty). */
    const int *rep;
    int *tri_shift;
    double tx, ty;
} ora_mesh;

static inline int node_rep(const ora_mesh *M, int n) { return M->rep ? M->rep[n] : n; }

/* ---------------------------------------------------------------- topology */

typedef struct { int a, b, t, m; } half_edge;

static int cmp_half(const void *p, const void *q)
{
    const half_edge *x = (const half_edge *)p, *y = (const half_edge *)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->t != y->t) return x->t < y->t ? -1 : 1;
    return x->m - y->m;
}

/* Orient, number edges, find neighbours, compute Whitney geometry.
 * Incidence C (face <- edge) is tri_edge/tri_sign (Sec. II.A, entries in {-1,0,1}).
 * Returns ne, or a negative error (degenerate triangle, non-manifold edge). */
int ora_mesh_build(ora_mesh *M, const int *tri_in)
{
    int nf = M->nf;
    const double *p = M->xy;
    for (int f = 0; f < nf; ++f) {
        int n0 = tri_in[3 * f], n1 = tri_in[3 * f + 1], n2 = tri_in[3 * f + 2];
        if (n0 < 0 || n1 < 0 || n2 < 0 || n0 >= M->nn || n1 >= M->nn || n2 >= M->nn) return ORA_EMESH;
        if (n0 == n1 || n1 == n2 || n0 == n2) return ORA_EMESH;
        double o = (p[2 * n1] - p[2 * n0]) * (p[2 * n2 + 1] - p[2 * n0 + 1])
                 - (p[2 * n2] - p[2 * n0]) * (p[2 * n1 + 1] - p[2 * n0 + 1]);
        if (o == 0.0) return ORA_EMESH;
        if (o < 0.0) { int t = n1; n1 = n2; n2 = t; }
        M->tri[3 * f] = n0; M->tri[3 * f + 1] = n1; M->tri[3 * f + 2] = n2;
    }
    half_edge *h = (half_edge *)malloc(sizeof(half_edge) * 3 * (size_t)nf);
    if (!h) return ORA_EINVAL;
    for (int f = 0; f < nf; ++f)
        for (int m = 0; m < 3; ++m) {
            /* edges join representative nodes: the two copies of a periodic edge are one edge */
            int u = node_rep(M, M->tri[3 * f + (m + 1) % 3]), v = node_rep(M, M->tri[3 * f + (m + 2) % 3]);
            if (u == v) { free(h); return ORA_EMESH; }      /* an edge joining a node to its own image */
            half_edge e;
            e.a = u < v ? u : v; e.b = u < v ? v : u; e.t = f; e.m = m;
            h[3 * f + m] = e;
        }
    qsort(h, 3 * (size_t)nf, sizeof(half_edge), cmp_half);
    int ne = 0;
    for (size_t k = 0; k < 3 * (size_t)nf;) {
        size_t k2 = k + 1;
        while (k2 < 3 * (size_t)nf && h[k2].a == h[k].a && h[k2].b == h[k].b) ++k2;
        if (k2 - k > 2) { free(h); return ORA_EMESH; }
        M->edge[2 * ne] = h[k].a; M->edge[2 * ne + 1] = h[k].b;
        M->edge_bnd[ne] = (k2 - k == 1);
        for (size_t r = k; r < k2; ++r) {
            int f = h[r].t, m = h[r].m;
            M->tri_edge[3 * f + m] = ne;
            /* local edge runs node m+1 -> m+2 */
            M->tri_sign[3 * f + m] = (node_rep(M, M->tri[3 * f + (m + 1) % 3]) == h[r].a) ? 1 : -1;
            M->tri_nb[3 * f + m] = -1;
            if (M->tri_shift) M->tri_shift[3 * f + m] = 0;
            if (k2 - k == 2) {
                const half_edge *o = &h[r == k ? k + 1 : k];
                M->tri_nb[3 * f + m] = o->t;
                if (M->tri_shift) {
                    /* the neighbour's copy of our node m+1 is its node o->m + 2 (opposite
                     * orientation); an image node lies one period beyond its representative */
                    int a1 = M->tri[3 * f + (m + 1) % 3];
                    int b2 = M->tri[3 * o->t + (o->m + 2) % 3];
                    M->tri_shift[3 * f + m] = (b2 != node_rep(M, b2)) - (a1 != node_rep(M, a1));
                }
            }
        }
        ++ne;
        k = k2;
    }
    free(h);
    M->ne = ne;
    /* Whitney geometry: lambda_m(r) = g_m . (r - r_{m+1}), g_m = grad lambda_m */
    for (int f = 0; f < nf; ++f) {
        double X[3], Y[3];
        for (int k = 0; k < 3; ++k) { X[k] = p[2 * M->tri[3 * f + k]]; Y[k] = p[2 * M->tri[3 * f + k] + 1]; }
        double d2A = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
        double inv = 1.0 / d2A;
        M->d2A[f] = d2A;
        M->inv2A[f] = inv;
        for (int m = 0; m < 3; ++m) {
            int a = (m + 1) % 3, b = (m + 2) % 3;
            M->gx[3 * f + m] = (Y[a] - Y[b]) * inv;
            M->gy[3 * f + m] = (X[b] - X[a]) * inv;
            M->nx_[3 * f + m] = X[m];
            M->ny_[3 * f + m] = Y[m];
        }
    }
    return ne;
}

/* Barycentric (Whitney 0-form, Sec. II.D) of point (x,y) in triangle f. */
static inline void lambdas(const ora_mesh *M, int f, double x, double y, double *l)
{
    for (int m = 0; m < 3; ++m) {
        int a = (m + 1) % 3;
        l[m] = M->gx[3 * f + m] * (x - M->nx_[3 * f + a]) + M->gy[3 * f + m] * (y - M->ny_[3 * f + a]);
    }
}

void ora_lambdas(const ora_mesh *M, int n, const int *cell, const double *x, const double *y, double *lam)
{
    for (int p = 0; p < n; ++p) lambdas(M, cell[p], x[p], y[p], lam + 3 * p);
}

/* Point location: the hint if all its lambdas are >= 0, else the lowest-index
 * triangle with all lambdas >= 0, else -1. */
int ora_locate(const ora_mesh *M, int n, const double *x, const double *y, const int *hint, int *cell)
{
    int bad = 0;
    for (int p = 0; p < n; ++p) {
        double l[3];
        int h = hint ? hint[p] : -1;
        if (h >= 0 && h < M->nf) {
            lambdas(M, h, x[p], y[p], l);
            if (l[0] >= 0.0 && l[1] >= 0.0 && l[2] >= 0.0) { cell[p] = h; continue; }
        }
        cell[p] = -1;
        for (int f = 0; f < M->nf; ++f) {
            lambdas(M, f, x[p], y[p], l);
            if (l[0] >= 0.0 && l[1] >= 0.0 && l[2] >= 0.0) { cell[p] = f; break; }
        }
        if (cell[p] < 0) ++bad;
    }
    return bad;
}

/* Electric field of the edge unknowns at points (Sec. II.B): in the triangle f
 * holding the point, E = sum_m s_m e_m (l_a grad l_b - l_b grad l_a) with
 * a = m+1, b = m+2 -- the interpolation of the particle gather, without
 * external fields.  Used for field probes along a line. */
void ora_field_at(const ora_mesh *M, const double *e, int n, const int *cell, const double *x, const double *y,
                  double *exy)
{
    for (int p = 0; p < n; ++p) {
        const int f = cell[p];
        double lam[3];
        lambdas(M, f, x[p], y[p], lam);
        const double *gx = M->gx + 3 * f, *gy = M->gy + 3 * f;
        double ex = 0.0, ey = 0.0;
        for (int m = 0; m < 3; ++m) {
            int a = (m + 1) % 3, b = (m + 2) % 3;
            double se = M->tri_sign[3 * f + m] * e[M->tri_edge[3 * f + m]];
            ex += se * (lam[a] * gx[b] - lam[b] * gx[a]);
            ey += se * (lam[a] * gy[b] - lam[b] * gy[a]);
        }
        exy[2 * p] = ex;
        exy[2 * p + 1] = ey;
    }
}

/* ------------------------------------------------------------ Hodge star */

/* Element matrices of [*eps] (Galerkin, eps0 * int W1_m . W1_n dA, Sec. II.A):
 * out[f][m][n] with global sign s_m s_n applied, for assembly by the caller.
 * Uses int lambda_a lambda_b dA = A (1 + delta_ab) / 12. */
void ora_hodge_eps_elements(const ora_mesh *M, double eps0, double *out)
{
    for (int f = 0; f < M->nf; ++f) {
        double A = 0.5 * M->d2A[f];
        const double *gx = M->gx + 3 * f, *gy = M->gy + 3 * f;
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) {
                int a = (m + 1) % 3, b = (m + 2) % 3, c = (n + 1) % 3, d = (n + 2) % 3;
                /* (l_a g_b - l_b g_a) . (l_c g_d - l_d g_c) */
                double Iac = A * (1.0 + (a == c)) / 12.0, Iad = A * (1.0 + (a == d)) / 12.0;
                double Ibc = A * (1.0 + (b == c)) / 12.0, Ibd = A * (1.0 + (b == d)) / 12.0;
                double gbgd = gx[b] * gx[d] + gy[b] * gy[d];
                double gbgc = gx[b] * gx[c] + gy[b] * gy[c];
                double gagd = gx[a] * gx[d] + gy[a] * gy[d];
                double gagc = gx[a] * gx[c] + gy[a] * gy[c];
                double v = Iac * gbgd - Iad * gbgc - Ibc * gagd + Ibd * gagc;
                out[9 * f + 3 * m + n] = eps0 * v * M->tri_sign[3 * f + m] * M->tri_sign[3 * f + n];
            }
    }
}

/* ------------------------------------------------------------------ SPAI */

/* Pattern P_k(j): vertices within k steps of j in the graph of A.  Returns the
 * count; ids written sorted ascending into out; mark/stamp is scratch. */
static int pattern(int n, const int *rp, const int *ci, int j, int k, int *out, int *mark, int stamp, int *tmp)
{
    (void)n;
    int cnt = 0;
    out[cnt++] = j; mark[j] = stamp;
    int lo = 0;
    for (int lev = 0; lev < k; ++lev) {
        int hi = cnt;
        for (int q = lo; q < hi; ++q) {
            int v = out[q];
            for (int r = rp[v]; r < rp[v + 1]; ++r) {
                int w = ci[r];
                if (mark[w] != stamp) { mark[w] = stamp; out[cnt++] = w; }
            }
        }
        lo = hi;
    }
    /* insertion sort is enough for the sizes involved, but use a counting merge */
    memcpy(tmp, out, sizeof(int) * cnt);
    for (int a = 1; a < cnt; ++a) {
        int v = tmp[a], b = a - 1;
        while (b >= 0 && tmp[b] > v) { tmp[b + 1] = tmp[b]; --b; }
        tmp[b + 1] = v;
    }
    memcpy(out, tmp, sizeof(int) * cnt);
    return cnt;
}

/* Total nnz of the level-k SPAI pattern (sum over columns of |P_k(j)|). */
long long ora_spai_count(int n, const int *rp, const int *ci, int k)
{
    int *mark = (int *)calloc(n, sizeof(int));
    int *buf = (int *)malloc(sizeof(int) * n), *tmp = (int *)malloc(sizeof(int) * n);
    long long tot = 0;
    for (int j = 0; j < n; ++j) tot += pattern(n, rp, ci, j, k, buf, mark, j + 1, tmp);
    free(mark); free(buf); free(tmp);
    return tot;
}

/* Sparse approximate inverse of the symmetric matrix A (CSR), Sec. II.A:
 * column j of M minimises || A m_j - e_j ||_2 with m_j supported on P_k(j).
 * The least-squares problem on rows P_{k+1}(j) is solved by Householder QR.
 * Output in CSC: colptr[n+1], rows[nnz], vals[nnz]. */
int ora_spai(int n, const int *rp, const int *ci, const double *v, int k,
             long long *colptr, int *rows, double *vals)
{
    int *mark = (int *)calloc(n, sizeof(int));
    int *markI = (int *)calloc(n, sizeof(int));
    int *J = (int *)malloc(sizeof(int) * n), *I = (int *)malloc(sizeof(int) * n);
    int *tmp = (int *)malloc(sizeof(int) * n);
    int *posI = (int *)malloc(sizeof(int) * n);
    long long off = 0;
    int status = ORA_OK;
    size_t cap = 0;
    double *Amat = NULL, *rhs = NULL;
    for (int j = 0; j < n; ++j) {
        int nJ = pattern(n, rp, ci, j, k, J, mark, j + 1, tmp);
        int nI = pattern(n, rp, ci, j, k + 1, I, markI, j + 1, tmp);
        size_t need = (size_t)nI * nJ;
        if (need > cap) {
            cap = need * 2;
            free(Amat);
            Amat = (double *)malloc(sizeof(double) * cap);
        }
        free(rhs);
        rhs = (double *)malloc(sizeof(double) * (size_t)nI);
        for (int a = 0; a < nI; ++a) posI[I[a]] = a;
        /* dense A[I,J], column-major: Amat[c*nI + r] */
        memset(Amat, 0, sizeof(double) * need);
        for (int c = 0; c < nJ; ++c) {
            int col = J[c];
            for (int r = rp[col]; r < rp[col + 1]; ++r)   /* A symmetric: row col == column col */
                Amat[(size_t)c * nI + posI[ci[r]]] = v[r];
        }
        for (int a = 0; a < nI; ++a) rhs[a] = (I[a] == j) ? 1.0 : 0.0;
        /* Householder QR, applied to rhs as we go */
        for (int c = 0; c < nJ; ++c) {
            double *col = Amat + (size_t)c * nI;
            double nrm = 0.0;
            for (int r = c; r < nI; ++r) nrm += col[r] * col[r];
            nrm = sqrt(nrm);
            if (nrm == 0.0) { status = ORA_EINVAL; continue; }
            double alpha = col[c] > 0 ? -nrm : nrm;
            double v0 = col[c] - alpha;
            /* Householder vector w = (v0, col[c+1..]) ; H = I - 2 w w^T / (w^T w) */
            double wtw = v0 * v0;
            for (int r = c + 1; r < nI; ++r) wtw += col[r] * col[r];
            if (wtw == 0.0) continue;
            for (int c2 = c + 1; c2 < nJ; ++c2) {
                double *o = Amat + (size_t)c2 * nI;
                double s = v0 * o[c];
                for (int r = c + 1; r < nI; ++r) s += col[r] * o[r];
                s = 2.0 * s / wtw;
                o[c] -= s * v0;
                for (int r = c + 1; r < nI; ++r) o[r] -= s * col[r];
            }
            {
                double s = v0 * rhs[c];
                for (int r = c + 1; r < nI; ++r) s += col[r] * rhs[r];
                s = 2.0 * s / wtw;
                rhs[c] -= s * v0;
                for (int r = c + 1; r < nI; ++r) rhs[r] -= s * col[r];
            }
            col[c] = alpha;
        }
        /* back substitution R m = Q^T e_j (first nJ rows) */
        colptr[j] = off;
        for (int c = nJ - 1; c >= 0; --c) {
            double s = rhs[c];
            for (int c2 = c + 1; c2 < nJ; ++c2) s -= Amat[(size_t)c2 * nI + c] * rhs[c2];
            rhs[c] = s / Amat[(size_t)c * nI + c];
        }
        for (int c = 0; c < nJ; ++c) { rows[off] = J[c]; vals[off] = rhs[c]; ++off; }
    }
    colptr[n] = off;
    free(mark); free(markI); free(J); free(I); free(tmp); free(posI); free(Amat); free(rhs);
    return status;
}

/* ------------------------------------------------------------ field update */

/* Faraday, Eq. (semi.dis.curl.1): b^{n+1/2} = b^{n-1/2} - dt C e^n. */
void ora_faraday(const ora_mesh *M, double dt, const double *e, const double *b_old, double *b_new)
{
    for (int f = 0; f < M->nf; ++f) {
        double ce = 0.0;
        for (int m = 0; m < 3; ++m) ce += M->tri_sign[3 * f + m] * e[M->tri_edge[3 * f + m]];
        b_new[f] = b_old[f] - dt * ce;
    }
}

/* r = C^T [*mu^-1] b - i over all edges; [*mu^-1] is diagonal 1/(mu0 A_f) for
 * the constant 2-D face form W2 = z/A_f. */
void ora_curl_h(const ora_mesh *M, double mu0, const double *b, const double *i_cur, double *r)
{
    for (int k = 0; k < M->ne; ++k) r[k] = 0.0;
    for (int f = 0; f < M->nf; ++f) {
        double hb = b[f] / (mu0 * (0.5 * M->d2A[f]));
        for (int m = 0; m < 3; ++m) r[M->tri_edge[3 * f + m]] += M->tri_sign[3 * f + m] * hb;
    }
    for (int k = 0; k < M->ne; ++k) r[k] -= i_cur[k];
}

/* Ampere, Eq. (semi.dis.curl.2) with the SPAI M ~ [*eps]^-1 over free edges:
 * e_free += dt * Minv r_free;  d += dt r (dual flux, all edges). */
void ora_ampere(int nfree, const int *free_ids, const long long *rp, const int *ci, const double *v,
                double dt, const double *r, double *e, double *d, int ne)
{
    for (int a = 0; a < nfree; ++a) {
        double s = 0.0;
        for (long long q = rp[a]; q < rp[a + 1]; ++q) s += v[q] * r[free_ids[ci[q]]];
        e[free_ids[a]] += dt * s;
    }
    if (d) for (int k = 0; k < ne; ++k) d[k] += dt * r[k];
}

/* ---------------------------------------------------------------- pushers */

static inline double gam(const double *u, double ic2)
{
    return sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * ic2);
}

static inline void cross(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Boris rotation u+ from u- with rotation vector t (Eqs. Boris.u2-u3). */
static inline void boris_rotate(const double *um, const double *t, double *up)
{
    double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double den = 1.0 + tt;
    double s[3] = { (2.0 * t[0]) / den, (2.0 * t[1]) / den, (2.0 * t[2]) / den };
    double c1[3], upr[3], c2[3];
    cross(um, t, c1);
    for (int k = 0; k < 3; ++k) upr[k] = um[k] + c1[k];
    cross(upr, s, c2);
    for (int k = 0; k < 3; ++k) up[k] = um[k] + c2[k];
}

/* One velocity update u^{n-1/2} -> u^{n+1/2}; returns gamma^{n+1/2} used for the
 * position update (Eq. eq.motion.dis). alpha = q dt / (2 m0). */
static double push(int pusher, double alpha, double c, double ic2,
                   const double *E, const double *B, double *u)
{
    double eps[3] = { alpha * E[0], alpha * E[1], alpha * E[2] };
    double beta[3] = { alpha * B[0], alpha * B[1], alpha * B[2] };
    double bb = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    if (pusher == ORA_VAY) {
        /* Sec. II.C(b) */
        double g0 = gam(u, ic2);
        double v[3] = { u[0] / g0, u[1] / g0, u[2] / g0 };
        double vb[3];
        cross(v, beta, vb);
        double un[3], up[3];
        for (int k = 0; k < 3; ++k) un[k] = u[k] + eps[k] + vb[k];
        for (int k = 0; k < 3; ++k) up[k] = un[k] + eps[k];
        double gp = gam(up, ic2);
        double sigma = gp * gp - bb;
        double ustar = (up[0] * beta[0] + up[1] * beta[1] + up[2] * beta[2]) / c;
        double gnew = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (bb + ustar * ustar))));
        double t[3] = { beta[0] / gnew, beta[1] / gnew, beta[2] / gnew };
        double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        double s = 1.0 / (1.0 + tt);
        double ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
        double uxt[3];
        cross(up, t, uxt);
        for (int k = 0; k < 3; ++k) u[k] = s * (up[k] + ut * t[k] + uxt[k]);
        return gnew;
    }
    double um[3] = { u[0] + eps[0], u[1] + eps[1], u[2] + eps[2] };   /* Eq. Boris.u1 */
    double gbar = gam(um, ic2);                                          /* Eq. gamma.middle */
    double t[3];
    if (pusher == ORA_HC) {
        double sigma = gbar * gbar - bb;
        double ustar = (beta[0] * um[0] + beta[1] * um[1] + beta[2] * um[2]) / c;
        double gh = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (bb + ustar * ustar))));
        for (int k = 0; k < 3; ++k) t[k] = beta[k] / gh;
    } else if (pusher == ORA_BORIS_TAN) {
        double nb = sqrt(bb);
        if (nb == 0.0) { t[0] = t[1] = t[2] = 0.0; }
        else {
            double tn = tan(nb / gbar);
            for (int k = 0; k < 3; ++k) t[k] = (beta[k] / nb) * tn;
        }
    } else {
        for (int k = 0; k < 3; ++k) t[k] = beta[k] / gbar;
    }
    double up[3];
    boris_rotate(um, t, up);                                             /* Eqs. Boris.u2-u3 */
    for (int k = 0; k < 3; ++k) u[k] = up[k] + eps[k];                   /* Eq. Boris.u4 */
    return gam(u, ic2);
}

/* ---------------------------------------------- gather, push, walk, deposit */

typedef struct {
    double dt, c, q, m;       /* species: superparticle charge and rest mass */
    double ext_ex, ext_ey, ext_bz;
    int pusher;
    int max_cross;
    /* applied fields that vary in space and time (a synchrocyclotron's magnet
     * and RF gap, Sec. III.A): in triangle f the external E is
     * (ext_amp * ext_w[2f]) * (ext_ex, ext_ey) and the external B_z is
     * ext_w[2f+1] * ext_bz; ext_w NULL = weights 1 */
    const double *ext_w;
    double ext_amp;
} ora_step_params;

/* Current of one sub-segment inside triangle f, Eq. (I.assign):
 * i_ab += (Q/dt) (l_a^s l_b^f - l_a^f l_b^s) for local edge m = (a,b). */
static inline void deposit(const ora_mesh *M, int f, const double *ls, const double *lf,
                           double qdt, double *i_acc, double *i_abs)
{
    for (int m = 0; m < 3; ++m) {
        int a = (m + 1) % 3, b = (m + 2) % 3;
        double d = ls[a] * lf[b] - lf[a] * ls[b];
        double v = qdt * d;
        int e = M->tri_edge[3 * f + m];
        i_acc[e] += M->tri_sign[3 * f + m] * v;
        if (i_abs) i_abs[e] += fabs(v);
    }
}

/* Advance n particles of one species by one step.
 * Gather (Sec. II.B) of E^n from e and B^n = (b^{n+1/2}+b^{n-1/2})/2 from the
 * face DoFs at r^n, push (Sec. II.C), r^{n+1} = r^n + dt u/gamma, walk the
 * segment across triangles and deposit the current of each sub-segment.
 * rec (optional): per particle up to rec_cap crossed edges (wall reflections
 * as -(edge+1)), rec_cnt[p] = number of crossings. */
int ora_particles(const ora_mesh *M, const ora_step_params *P,
                  const double *e, const double *b_old, const double *b_new,
                  int n, double *x, double *y, double *ux, double *uy, double *uz, int *cell,
                  double *i_acc, double *i_abs, int rec_cap, int *rec_cnt, int *rec)
{
    const double ic2 = 1.0 / (P->c * P->c);
    const double alpha = P->q * P->dt / (2.0 * P->m);
    const double qdt = P->q / P->dt;
    int status = ORA_OK;
    for (int p = 0; p < n; ++p) {
        int f = cell[p];
        double lam[3];
        lambdas(M, f, x[p], y[p], lam);
        /* gather E^n: sum_m s_m e_m (l_a grad l_b - l_b grad l_a) */
        const double *gx = M->gx + 3 * f, *gy = M->gy + 3 * f;
        double E[3] = { 0.0, 0.0, 0.0 };
        for (int m = 0; m < 3; ++m) {
            int a = (m + 1) % 3, b = (m + 2) % 3;
            double se = M->tri_sign[3 * f + m] * e[M->tri_edge[3 * f + m]];
            double wx = lam[a] * gx[b] - lam[b] * gx[a];
            double wy = lam[a] * gy[b] - lam[b] * gy[a];
            E[0] += se * wx;
            E[1] += se * wy;
        }
        const double we = P->ext_w ? P->ext_w[2 * f] : 1.0, wb = P->ext_w ? P->ext_w[2 * f + 1] : 1.0;
        const double se = P->ext_amp * we;
        E[0] += se * P->ext_ex;
        E[1] += se * P->ext_ey;
        double B[3] = { 0.0, 0.0, (b_new[f] + b_old[f]) * M->inv2A[f] + wb * P->ext_bz };
        double u[3] = { ux[p], uy[p], uz[p] };
        double g = push(P->pusher, alpha, P->c, ic2, E, B, u);
        double ig = 1.0 / g;
        double xs = x[p], ys = y[p];
        double xf = xs + (u[0] * ig) * P->dt;
        double yf = ys + (u[1] * ig) * P->dt;
        /* walk */
        double lin[3] = { lam[0], lam[1], lam[2] };
        int min = -1, ncross = 0;
        double tin = 0.0;
        for (;;) {
            double ls[3], lf[3];
            lambdas(M, f, xs, ys, ls);
            lambdas(M, f, xf, yf, lf);
            int best = -1;
            double tb = 0.0;
            for (int k = 0; k < 3; ++k) {
                if (k == min) continue;
                if (lf[k] < 0.0) {
                    double den = ls[k] - lf[k];
                    double t = den > 0.0 ? ls[k] / den : tin;
                    if (t < tin) t = tin;
                    if (best < 0 || t < tb) { best = k; tb = t; }
                }
            }
            if (best < 0) {
                deposit(M, f, lin, lf, qdt, i_acc, i_abs);
                break;
            }
            double lout[3];
            for (int k = 0; k < 3; ++k) lout[k] = ls[k] + tb * (lf[k] - ls[k]);
            lout[best] = 0.0;
            deposit(M, f, lin, lout, qdt, i_acc, i_abs);
            int eg = M->tri_edge[3 * f + best];
            if (ncross >= P->max_cross) {
                /* stop on the crossing point; flag the error */
                xf = xs + tb * (xf - xs);
                yf = ys + tb * (yf - ys);
                status = ORA_EWALK;
                break;
            }
            int nb = M->tri_nb[3 * f + best];
            if (rec && ncross < rec_cap) rec[(size_t)p * rec_cap + ncross] = nb < 0 ? -(eg + 1) : eg;
            ++ncross;
            if (nb < 0) {
                /* PEC wall: specular reflection of the remaining segment and of u */
                double xw = xs + tb * (xf - xs), yw = ys + tb * (yf - ys);
                double gxb = gx[best], gyb = gy[best];
                double gg = gxb * gxb + gyb * gyb;
                double pr = ((xf - xw) * gxb + (yf - yw) * gyb) / gg;
                xf = xf - 2.0 * pr * gxb;
                yf = yf - 2.0 * pr * gyb;
                double pu = (u[0] * gxb + u[1] * gyb) / gg;
                u[0] = u[0] - 2.0 * pu * gxb;
                u[1] = u[1] - 2.0 * pu * gyb;
                xs = xw; ys = yw;
                tin = 0.0;
                min = best;
                for (int k = 0; k < 3; ++k) lin[k] = lout[k];
            } else {
                int m2 = 0;
                while (m2 < 3 && M->tri_edge[3 * nb + m2] != eg) ++m2;
                if (m2 == 3) { status = ORA_EMESH; break; }
                /* periodic wall: the rest of the segment continues from the other copy */
                int sc = M->tri_shift ? M->tri_shift[3 * f + best] : 0;
                if (sc != 0) {
                    xs = xs + sc * M->tx; ys = ys + sc * M->ty;
                    xf = xf + sc * M->tx; yf = yf + sc * M->ty;
                }
                double l2[3];
                l2[m2] = 0.0;
                l2[(m2 + 1) % 3] = lout[(best + 2) % 3];
                l2[(m2 + 2) % 3] = lout[(best + 1) % 3];
                for (int k = 0; k < 3; ++k) lin[k] = l2[k];
                f = nb;
                min = m2;
                tin = tb;
                gx = M->gx + 3 * f; gy = M->gy + 3 * f;
            }
        }
        if (rec_cnt) rec_cnt[p] = ncross;
        x[p] = xf; y[p] = yf;
        ux[p] = u[0]; uy[p] = u[1]; uz[p] = u[2];
        cell[p] = f;
    }
    return status;
}

/* Nodal charge, Eq. (scatter.charge.assign): q_i += Q lambda_i(r_p). */
void ora_charge(const ora_mesh *M, double Q, int n, const double *x, const double *y,
                const int *cell, double *q_node)
{
    for (int p = 0; p < n; ++p) {
        double l[3];
        int f = cell[p];
        lambdas(M, f, x[p], y[p], l);
        for (int k = 0; k < 3; ++k) q_node[node_rep(M, M->tri[3 * f + k])] += Q * l[k];
    }
}

/* Push only (no mesh): used by the closed-form pusher pins. */
double ora_push_only(int pusher, double alpha, double c, const double *E, const double *B, double *u)
{
    return push(pusher, alpha, c, 1.0 / (c * c), E, B, u);
}
