// Host-side setup of one mesh instance: validation, counter-clockwise
// orientation, edge numbering and incidence (Sec. II.A), Whitney geometry,
// the Galerkin Hodge matrix [*eps] and its sparse approximate inverse.
//
// Compiled with -ffp-contract=off: the triangle geometry must round exactly
// as written, because the FP64 particle kernels evaluate the same formulas
// and plain-FP64 runs are compared bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <unordered_map>

#include "fetdpic_internal.h"
#include "fetdpic.h"

namespace fetdpic {

static inline long long pair_key(int a, int b)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return ((long long)lo << 32) | (unsigned)hi;
}

// Position of cell (x, y) of a 2^order x 2^order grid along the Hilbert curve
// (the curve's recursive quadrant rule, one level per bit from the top).
static unsigned long long hilbert_index(unsigned x, unsigned y, int order)
{
    const unsigned n = 1u << order;
    unsigned long long d = 0;
    for (unsigned s = n >> 1; s > 0; s >>= 1) {
        const unsigned rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += (unsigned long long)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {                       // reflect / transpose the quadrant so the curve stays continuous
            if (rx == 1) { x = n - 1 - x; y = n - 1 - y; }
            std::swap(x, y);
        }
    }
    return d;
}

std::vector<int> hilbert_order(int nn, const double *xy, int nf, const int *tri)
{
    std::vector<int> perm(nf);
    for (int f = 0; f < nf; ++f) perm[f] = f;
    if (nf < 2) return perm;
    double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
    std::vector<double> c(2 * (size_t)nf);
    for (int f = 0; f < nf; ++f)
        for (int d = 0; d < 2; ++d) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) {
                const int n = tri[3 * f + k];
                v += (n >= 0 && n < nn) ? xy[2 * n + d] : 0.0;
            }
            c[2 * f + d] = v / 3.0;
            lo[d] = std::min(lo[d], c[2 * f + d]);
            hi[d] = std::max(hi[d], c[2 * f + d]);
        }
    const double span = std::max(hi[0] - lo[0], hi[1] - lo[1]);
    const int order = 16;
    const double scale = span > 0 ? ((1 << order) - 1) / span : 0.0;
    std::vector<unsigned long long> key(nf);
    for (int f = 0; f < nf; ++f) {
        const unsigned x = (unsigned)((c[2 * f] - lo[0]) * scale), y = (unsigned)((c[2 * f + 1] - lo[1]) * scale);
        key[f] = hilbert_index(x, y, order);
    }
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return key[a] < key[b]; });
    return perm;
}

int build_mesh(HostMesh &M, int nn, const double *xy, int nf, const int *tri_caller,
               int ne_in, const int *edges_in, const int *tags_in,
               int n_per, const int *per_nodes, double tx, double ty, std::string &msg)
{
    if (nn <= 0 || nf <= 0 || !xy || !tri_caller) { msg = "empty mesh"; return FETDPIC_EINVAL; }
    M.nn = nn; M.nf = nf;
    // triangles are stored along the Hilbert curve; messages name the caller's indices
    M.perm = hilbert_order(nn, xy, nf, tri_caller);
    M.inv.assign(nf, 0);
    for (int k = 0; k < nf; ++k) M.inv[M.perm[k]] = k;
    std::vector<int> tri_store(3 * (size_t)nf);
    for (int k = 0; k < nf; ++k)
        for (int j = 0; j < 3; ++j) tri_store[3 * (size_t)k + j] = tri_caller[3 * (size_t)M.perm[k] + j];
    const int *tri_in = tri_store.data();
    M.xy.assign(xy, xy + 2 * (size_t)nn);
    // periodic walls: each image node becomes its representative (Sec. III.C strip)
    M.rep.resize(nn);
    for (int n = 0; n < nn; ++n) M.rep[n] = n;
    M.periodic = n_per > 0;
    M.tx = tx; M.ty = ty;
    if (n_per < 0 || (n_per > 0 && !per_nodes)) { msg = "bad periodic node list"; return FETDPIC_EINVAL; }
    if (M.periodic) {
        if (edges_in || tags_in) { msg = "periodic walls need derived edges and tags"; return FETDPIC_EINVAL; }
        if (!(std::isfinite(tx) && std::isfinite(ty)) || (tx == 0.0 && ty == 0.0)) {
            msg = "periodic walls need a nonzero period"; return FETDPIC_EINVAL;
        }
        double ext = std::fabs(tx) + std::fabs(ty);
        for (int n = 0; n < nn; ++n) ext = std::max(ext, std::max(std::fabs(xy[2 * n]), std::fabs(xy[2 * n + 1])));
        for (int k = 0; k < n_per; ++k) {
            const int a = per_nodes[2 * k], b = per_nodes[2 * k + 1];
            if (a < 0 || b < 0 || a >= nn || b >= nn || a == b) { msg = "periodic pair " + std::to_string(k) + " out of range"; return FETDPIC_EINVAL; }
            if (M.rep[b] != b || M.rep[a] != a) { msg = "node in more than one periodic pair role"; return FETDPIC_EINVAL; }
            if (std::fabs(xy[2 * b] - xy[2 * a] - tx) > 1e-9 * ext || std::fabs(xy[2 * b + 1] - xy[2 * a + 1] - ty) > 1e-9 * ext) {
                msg = "periodic pair " + std::to_string(k) + ": node b is not node a moved by the period"; return FETDPIC_EMESH;
            }
            M.rep[b] = a;
        }
    }
    M.tri.resize(3 * (size_t)nf);
    for (int f = 0; f < nf; ++f) {
        int v[3] = {tri_in[3 * f], tri_in[3 * f + 1], tri_in[3 * f + 2]};
        for (int k = 0; k < 3; ++k)
            if (v[k] < 0 || v[k] >= nn) { msg = "triangle " + std::to_string(M.perm[f]) + " has a node id out of range"; return FETDPIC_EMESH; }
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) { msg = "triangle " + std::to_string(M.perm[f]) + " repeats a node"; return FETDPIC_EMESH; }
        const double *p0 = &xy[2 * v[0]], *p1 = &xy[2 * v[1]], *p2 = &xy[2 * v[2]];
        double o = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]);
        if (!(o != 0.0)) { msg = "triangle " + std::to_string(M.perm[f]) + " has zero area"; return FETDPIC_EMESH; }
        if (o < 0.0) std::swap(v[1], v[2]);
        for (int k = 0; k < 3; ++k) M.tri[3 * f + k] = v[k];
    }

    // edge numbering: derived = sorted unique (lo, hi) pairs; given = caller's order
    std::vector<long long> keys;
    std::unordered_map<long long, int> given;
    if (edges_in) {
        if (ne_in <= 0) { msg = "n_edges must be > 0 with an edge list"; return FETDPIC_EINVAL; }
        M.ne = ne_in;
        M.edge.assign(edges_in, edges_in + 2 * (size_t)ne_in);
        given.reserve(2 * (size_t)ne_in);
        for (int e = 0; e < ne_in; ++e) {
            int a = edges_in[2 * e], b = edges_in[2 * e + 1];
            if (a < 0 || b < 0 || a >= nn || b >= nn || a == b) { msg = "bad edge " + std::to_string(e); return FETDPIC_EMESH; }
            if (!given.emplace(pair_key(a, b), e).second) { msg = "duplicate edge " + std::to_string(e); return FETDPIC_EMESH; }
        }
    } else {
        keys.reserve(3 * (size_t)nf);
        for (int f = 0; f < nf; ++f)
            for (int m = 0; m < 3; ++m) {
                const int a = M.rep[M.tri[3 * f + (m + 1) % 3]], b = M.rep[M.tri[3 * f + (m + 2) % 3]];
                if (a == b) { msg = "triangle " + std::to_string(M.perm[f]) + " joins a node to its periodic image"; return FETDPIC_EMESH; }
                keys.push_back(pair_key(a, b));
            }
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
        M.ne = (int)keys.size();
        M.edge.resize(2 * (size_t)M.ne);
        for (int e = 0; e < M.ne; ++e) { M.edge[2 * e] = (int)(keys[e] >> 32); M.edge[2 * e + 1] = (int)(keys[e] & 0xffffffffLL); }
    }
    const int ne = M.ne;
    M.tedge.assign(3 * (size_t)nf, -1);
    M.tsign.assign(3 * (size_t)nf, 0);
    M.tnb.assign(3 * (size_t)nf, -1);
    M.tnbm.assign(3 * (size_t)nf, -1);
    M.efac.assign(2 * (size_t)ne, -1);
    M.efsign.assign(2 * (size_t)ne, 0);
    for (int f = 0; f < nf; ++f)
        for (int m = 0; m < 3; ++m) {
            int a = M.rep[M.tri[3 * f + (m + 1) % 3]], b = M.rep[M.tri[3 * f + (m + 2) % 3]];
            long long k = pair_key(a, b);
            int e;
            if (edges_in) {
                auto it = given.find(k);
                if (it == given.end()) { msg = "edge list misses an edge of triangle " + std::to_string(M.perm[f]); return FETDPIC_EMESH; }
                e = it->second;
            } else {
                e = (int)(std::lower_bound(keys.begin(), keys.end(), k) - keys.begin());
            }
            M.tedge[3 * f + m] = e;
            M.tsign[3 * f + m] = (M.edge[2 * e] == a) ? 1 : -1;
            if (M.efac[2 * e] < 0) { M.efac[2 * e] = f; M.efsign[2 * e] = M.tsign[3 * f + m]; }
            else if (M.efac[2 * e + 1] < 0) { M.efac[2 * e + 1] = f; M.efsign[2 * e + 1] = M.tsign[3 * f + m]; }
            else { msg = "edge shared by more than two triangles"; return FETDPIC_EMESH; }
        }
    for (int e = 0; e < ne; ++e) {
        if (M.efac[2 * e] < 0) { msg = "edge " + std::to_string(e) + " belongs to no triangle"; return FETDPIC_EMESH; }
        if (M.efac[2 * e + 1] >= 0 && M.efsign[2 * e] == M.efsign[2 * e + 1]) {
            msg = "inconsistent orientation across edge " + std::to_string(e); return FETDPIC_EMESH;
        }
    }
    M.tshift.assign(3 * (size_t)nf, 0);
    for (int f = 0; f < nf; ++f)
        for (int m = 0; m < 3; ++m) {
            int e = M.tedge[3 * f + m];
            int g = M.efac[2 * e] == f ? M.efac[2 * e + 1] : M.efac[2 * e];
            M.tnb[3 * f + m] = g;
            if (g >= 0)
                for (int m2 = 0; m2 < 3; ++m2) if (M.tedge[3 * g + m2] == e) M.tnbm[3 * f + m] = m2;
            if (g >= 0 && M.periodic) {
                // the neighbour's copy of our node m+1 is its node m2+2; an image node lies one
                // period beyond its representative
                const int a1 = M.tri[3 * f + (m + 1) % 3];
                const int b2 = M.tri[3 * g + (M.tnbm[3 * f + m] + 2) % 3];
                M.tshift[3 * f + m] = (signed char)((M.rep[b2] != b2) - (M.rep[a1] != a1));
            }
        }
    M.pec.assign(ne, 0);
    for (int e = 0; e < ne; ++e) {
        if (tags_in) M.pec[e] = tags_in[e] != 0;
        else M.pec[e] = M.efac[2 * e + 1] < 0;
    }
    // Whitney geometry (Sec. II.B): grad lambda_m = (Y_{m+1} - Y_{m+2}, X_{m+2} - X_{m+1}) / (2A)
    M.d2A.resize(nf); M.inv2A.resize(nf);
    M.gx.resize(3 * (size_t)nf); M.gy.resize(3 * (size_t)nf); M.X.resize(3 * (size_t)nf); M.Y.resize(3 * (size_t)nf);
    for (int f = 0; f < nf; ++f) {
        double X[3], Y[3];
        for (int k = 0; k < 3; ++k) { X[k] = xy[2 * M.tri[3 * f + k]]; Y[k] = xy[2 * M.tri[3 * f + k] + 1]; }
        const double d2A = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
        const double inv = 1.0 / d2A;
        M.d2A[f] = d2A; M.inv2A[f] = inv;
        for (int m = 0; m < 3; ++m) {
            const int a = (m + 1) % 3, b = (m + 2) % 3;
            M.gx[3 * f + m] = (Y[a] - Y[b]) * inv;
            M.gy[3 * f + m] = (X[b] - X[a]) * inv;
            M.X[3 * f + m] = X[m];
            M.Y[3 * f + m] = Y[m];
        }
    }
    // edge vectors from the geometry of a triangle holding the edge (the two
    // stored nodes of a periodic edge may be a period apart)
    M.evec.assign(2 * (size_t)ne, 0.0);
    for (int f = 0; f < nf; ++f)
        for (int m = 0; m < 3; ++m) {
            const int e = M.tedge[3 * f + m];
            if (M.efac[2 * e] != f) continue;
            const int a = (m + 1) % 3, b = (m + 2) % 3;
            const double sg = M.tsign[3 * f + m];
            M.evec[2 * e] = sg * (M.X[3 * f + b] - M.X[3 * f + a]);
            M.evec[2 * e + 1] = sg * (M.Y[3 * f + b] - M.Y[3 * f + a]);
        }
    M.free_edges.clear();
    for (int e = 0; e < ne; ++e) if (!M.pec[e]) M.free_edges.push_back(e);
    return FETDPIC_OK;
}

int electrostatic_solve(const HostMesh &M, const std::vector<double> &q, std::vector<double> &de,
                        int &iterations, double &rel_residual, std::string &msg)
{
    const int nn = M.nn, ne = M.ne;
    if ((int)q.size() != nn) { msg = "charge size"; return FETDPIC_EINVAL; }
    if (M.h_rp.empty()) { msg = "Hodge matrix not built"; return FETDPIC_ESTATE; }
    // unknowns: nodes that bound a free edge and no PEC edge (images own no edge)
    std::vector<char> has_free(nn, 0), on_pec(nn, 0);
    for (int e = 0; e < ne; ++e) {
        const int a = M.edge[2 * e], b = M.edge[2 * e + 1];
        if (M.pec[e]) { on_pec[a] = on_pec[b] = 1; }
        else { has_free[a] = has_free[b] = 1; }
    }
    std::vector<char> unk(nn);
    bool any_pec = false;
    for (int n = 0; n < nn; ++n) { unk[n] = has_free[n] && !on_pec[n]; any_pec = any_pec || on_pec[n]; }
    if (!any_pec) { msg = "the electrostatic solve needs a PEC wall (the potential is fixed there)"; return FETDPIC_ESTATE; }
    // K phi = G^T [*eps] (G phi) over free edges, phi = 0 off the unknowns
    std::vector<double> g(ne), h(ne);
    auto apply = [&](const std::vector<double> &phi, std::vector<double> &out) {
        for (int e = 0; e < ne; ++e) g[e] = M.pec[e] ? 0.0 : phi[M.edge[2 * e + 1]] - phi[M.edge[2 * e]];
        for (int e = 0; e < ne; ++e) {
            double s = 0.0;
            if (!M.pec[e])
                for (long long k = M.h_rp[e]; k < M.h_rp[e + 1]; ++k) s += M.h_v[k] * g[M.h_ci[k]];
            h[e] = s;
        }
        std::fill(out.begin(), out.end(), 0.0);
        for (int e = 0; e < ne; ++e) {
            out[M.edge[2 * e + 1]] += h[e];
            out[M.edge[2 * e]] -= h[e];
        }
        for (int n = 0; n < nn; ++n) if (!unk[n]) out[n] = 0.0;
    };
    // Jacobi: diag K ~ sum over incident free edges of [*eps]_ee
    std::vector<double> dg(nn, 0.0);
    for (int e = 0; e < ne; ++e) {
        if (M.pec[e]) continue;
        double dee = 0.0;
        for (long long k = M.h_rp[e]; k < M.h_rp[e + 1]; ++k) if (M.h_ci[k] == e) dee = M.h_v[k];
        dg[M.edge[2 * e]] += dee; dg[M.edge[2 * e + 1]] += dee;
    }
    std::vector<double> x(nn, 0.0), r(nn), z(nn), pv(nn), Ap(nn);
    double bn = 0.0;
    for (int n = 0; n < nn; ++n) { r[n] = unk[n] ? q[n] : 0.0; bn += r[n] * r[n]; }
    bn = std::sqrt(bn);
    iterations = 0; rel_residual = 0.0;
    de.assign(ne, 0.0);
    if (bn == 0.0) return FETDPIC_OK;
    for (int n = 0; n < nn; ++n) z[n] = unk[n] && dg[n] > 0 ? r[n] / dg[n] : 0.0;
    pv = z;
    double rz = 0.0;
    for (int n = 0; n < nn; ++n) rz += r[n] * z[n];
    const int max_it = 20 * nn + 100;
    double rn = bn;
    for (int it = 1; it <= max_it; ++it) {
        apply(pv, Ap);
        double pAp = 0.0;
        for (int n = 0; n < nn; ++n) pAp += pv[n] * Ap[n];
        if (!(pAp > 0.0)) { msg = "electrostatic solve: matrix not positive definite"; return FETDPIC_EMESH; }
        const double alpha = rz / pAp;
        rn = 0.0;
        for (int n = 0; n < nn; ++n) { x[n] += alpha * pv[n]; r[n] -= alpha * Ap[n]; rn += r[n] * r[n]; }
        rn = std::sqrt(rn);
        iterations = it;
        if (rn <= 1e-14 * bn) break;
        for (int n = 0; n < nn; ++n) z[n] = unk[n] && dg[n] > 0 ? r[n] / dg[n] : 0.0;
        double rz2 = 0.0;
        for (int n = 0; n < nn; ++n) rz2 += r[n] * z[n];
        const double beta = rz2 / rz;
        rz = rz2;
        for (int n = 0; n < nn; ++n) pv[n] = z[n] + beta * pv[n];
    }
    rel_residual = rn / bn;
    if (rel_residual > 1e-12) { msg = "electrostatic solve did not converge"; return FETDPIC_EMESH; }
    for (int e = 0; e < ne; ++e) de[e] = M.pec[e] ? 0.0 : -(x[M.edge[2 * e + 1]] - x[M.edge[2 * e]]);
    return FETDPIC_OK;
}

void host_lambdas(const HostMesh &M, int f, double x, double y, double *l)
{
    for (int m = 0; m < 3; ++m) {
        const int a = (m + 1) % 3;
        l[m] = M.gx[3 * f + m] * (x - M.X[3 * f + a]) + M.gy[3 * f + m] * (y - M.Y[3 * f + a]);
    }
}

int host_locate(const HostMesh &M, double x, double y, int hint)
{
    // hint and the scan are in the caller's triangle order; the result is the stored index
    double l[3];
    if (hint >= 0 && hint < M.nf) {
        const int f = M.inv[hint];
        host_lambdas(M, f, x, y, l);
        if (l[0] >= 0.0 && l[1] >= 0.0 && l[2] >= 0.0) return f;
    }
    for (int k = 0; k < M.nf; ++k) {
        const int f = M.inv[k];
        host_lambdas(M, f, x, y, l);
        if (l[0] >= 0.0 && l[1] >= 0.0 && l[2] >= 0.0) return f;
    }
    return -1;
}

// [*eps]_{jk} = eps0 sum_T int_T W1_j . W1_k dA, Galerkin edge mass matrix.
// In a triangle W1_m = l_a grad l_b - l_b grad l_a and
// int l_p l_q dA = A (1 + [p == q]) / 12.
int build_hodge(HostMesh &M, double eps0, std::string &msg)
{
    (void)msg;
    const int nf = M.nf, ne = M.ne;
    std::vector<std::vector<std::pair<int, double>>> rows(ne);
    for (int f = 0; f < nf; ++f) {
        const double A = 0.5 * M.d2A[f];
        const double *gx = &M.gx[3 * f], *gy = &M.gy[3 * f];
        double G[3][3];
        for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) G[p][q] = gx[p] * gx[q] + gy[p] * gy[q];
        auto I = [&](int p, int q) { return (p == q ? 2.0 : 1.0) * A / 12.0; };
        for (int m = 0; m < 3; ++m) {
            const int a = (m + 1) % 3, b = (m + 2) % 3;
            for (int n = 0; n < 3; ++n) {
                const int c = (n + 1) % 3, d = (n + 2) % 3;
                double v = I(a, c) * G[b][d] - I(a, d) * G[b][c] - I(b, c) * G[a][d] + I(b, d) * G[a][c];
                v *= eps0 * M.tsign[3 * f + m] * M.tsign[3 * f + n];
                rows[M.tedge[3 * f + m]].push_back({M.tedge[3 * f + n], v});
            }
        }
    }
    auto compress = [](std::vector<std::pair<int, double>> &r) {
        std::sort(r.begin(), r.end(), [](auto &x, auto &y) { return x.first < y.first; });
        size_t w = 0;
        for (size_t k = 0; k < r.size(); ++k) {
            if (w > 0 && r[w - 1].first == r[k].first) r[w - 1].second += r[k].second;
            else r[w++] = r[k];
        }
        r.resize(w);
    };
    M.h_rp.assign(ne + 1, 0); M.h_ci.clear(); M.h_v.clear();
    for (int e = 0; e < ne; ++e) {
        compress(rows[e]);
        for (auto &kv : rows[e]) { M.h_ci.push_back(kv.first); M.h_v.push_back(kv.second); }
        M.h_rp[e + 1] = (long long)M.h_ci.size();
    }
    // free-edge restriction with free-edge indices
    std::vector<int> fidx(ne, -1);
    for (size_t a = 0; a < M.free_edges.size(); ++a) fidx[M.free_edges[a]] = (int)a;
    M.a_rp.assign(M.free_edges.size() + 1, 0); M.a_ci.clear(); M.a_v.clear();
    for (size_t a = 0; a < M.free_edges.size(); ++a) {
        int e = M.free_edges[a];
        for (long long q = M.h_rp[e]; q < M.h_rp[e + 1]; ++q)
            if (fidx[M.h_ci[q]] >= 0) { M.a_ci.push_back(fidx[M.h_ci[q]]); M.a_v.push_back(M.h_v[q]); }
        M.a_rp[a + 1] = (long long)M.a_ci.size();
    }
    return FETDPIC_OK;
}

// Cholesky solve of a small dense SPD system (in place, row-major n x n).
static bool chol_solve(std::vector<double> &G, std::vector<double> &rhs, int n)
{
    for (int j = 0; j < n; ++j) {
        double s = G[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= G[(size_t)j * n + k] * G[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double d = std::sqrt(s);
        G[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = G[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= G[(size_t)i * n + k] * G[(size_t)j * n + k];
            G[(size_t)i * n + j] = t / d;
        }
    }
    for (int i = 0; i < n; ++i) {
        double t = rhs[i];
        for (int k = 0; k < i; ++k) t -= G[(size_t)i * n + k] * rhs[k];
        rhs[i] = t / G[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = rhs[i];
        for (int k = i + 1; k < n; ++k) t -= G[(size_t)k * n + i] * rhs[k];
        rhs[i] = t / G[(size_t)i * n + i];
    }
    return true;
}

// Sparse approximate inverse (Sec. II.A): column j of M minimises
// ||A m - e_j||_2 over m supported on the level-`level` neighbourhood J of j in
// the graph of A.  With A symmetric and every nonzero row of A[:, J] kept,
// the normal equations read (A^2)[J, J] m = A[J, j]; they are solved by
// Cholesky.  M is then symmetrised.  level < 0: exact dense inverse.
int build_spai(HostMesh &M, int level, std::string &msg)
{
    const int n = (int)M.free_edges.size();
    std::vector<std::vector<int>> colJ(n);
    std::vector<std::vector<double>> colV(n);
    if (n == 0) { M.m_rp.assign(1, 0); M.m_ci.clear(); M.m_v.clear(); return FETDPIC_OK; }
    if (level < 0) {
        if (n > 4096) { msg = "exact inverse needs <= 4096 free edges"; return FETDPIC_EINVAL; }
        std::vector<double> G((size_t)n * n, 0.0);
        for (int a = 0; a < n; ++a)
            for (long long q = M.a_rp[a]; q < M.a_rp[a + 1]; ++q) G[(size_t)a * n + M.a_ci[q]] = M.a_v[q];
        for (int j = 0; j < n; ++j) {
            std::vector<double> Gc = G, rhs(n, 0.0);
            rhs[j] = 1.0;
            if (!chol_solve(Gc, rhs, n)) { msg = "[*eps] not positive definite"; return FETDPIC_EMESH; }
            for (int a = 0; a < n; ++a) { colJ[j].push_back(a); colV[j].push_back(rhs[a]); }
        }
    } else {
        const int k = level == 0 ? 2 : level;
        int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        std::vector<int> fail(nth, 0);
        auto work = [&](int tid) {
            std::vector<int> stamp(n, -1), pos(n, -1), J, frontier, next;
            std::vector<double> G, rhs;
            for (int j = tid; j < n; j += nth) {
                J.clear(); frontier.clear();
                J.push_back(j); frontier.push_back(j); stamp[j] = j;
                for (int lev = 0; lev < k; ++lev) {
                    next.clear();
                    for (int v : frontier)
                        for (long long q = M.a_rp[v]; q < M.a_rp[v + 1]; ++q) {
                            int w = M.a_ci[q];
                            if (stamp[w] != j) { stamp[w] = j; J.push_back(w); next.push_back(w); }
                        }
                    frontier.swap(next);
                }
                std::sort(J.begin(), J.end());
                const int nJ = (int)J.size();
                for (int c = 0; c < nJ; ++c) pos[J[c]] = c;
                // (A^2)[J,J] = sum over rows i of A[i,J]^T A[i,J]; rows are the union of patterns of J
                G.assign((size_t)nJ * nJ, 0.0);
                rhs.assign(nJ, 0.0);
                // iterate rows i reachable from J: for each column c in J, A[i, J[c]] = A[J[c], i]
                // accumulate via row lists: for each row i, its entries inside J
                std::vector<std::pair<int, double>> rowent;
                std::vector<int> rows;
                for (int c = 0; c < nJ; ++c)
                    for (long long q = M.a_rp[J[c]]; q < M.a_rp[J[c] + 1]; ++q) rows.push_back(M.a_ci[q]);
                std::sort(rows.begin(), rows.end());
                rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
                for (int i : rows) {
                    rowent.clear();
                    for (long long q = M.a_rp[i]; q < M.a_rp[i + 1]; ++q) {
                        int w = M.a_ci[q];
                        if (stamp[w] == j && pos[w] >= 0 && pos[w] < nJ && J[pos[w]] == w) rowent.push_back({pos[w], M.a_v[q]});
                    }
                    for (auto &x : rowent)
                        for (auto &y : rowent) G[(size_t)x.first * nJ + y.first] += x.second * y.second;
                    if (i == j) for (auto &x : rowent) rhs[x.first] += x.second;
                }
                if (!chol_solve(G, rhs, nJ)) { fail[tid] = 1; }
                colJ[j] = J;
                colV[j].assign(rhs.begin(), rhs.end());
                for (int c = 0; c < nJ; ++c) pos[J[c]] = -1;
            }
        };
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t) th.emplace_back(work, t);
        for (auto &t : th) t.join();
        for (int f : fail) if (f) { msg = "SPAI normal equations not positive definite"; return FETDPIC_EMESH; }
    }
    // symmetrise: M = (M + M^T)/2, rows over free edges, columns as edge ids
    std::vector<std::vector<std::pair<int, double>>> rows(n);
    for (int j = 0; j < n; ++j)
        for (size_t c = 0; c < colJ[j].size(); ++c) {
            const int i = colJ[j][c];
            const double v = 0.5 * colV[j][c];
            rows[i].push_back({j, v});
            rows[j].push_back({i, v});
        }
    M.m_rp.assign(n + 1, 0); M.m_ci.clear(); M.m_v.clear();
    for (int i = 0; i < n; ++i) {
        auto &r = rows[i];
        std::sort(r.begin(), r.end(), [](auto &x, auto &y) { return x.first < y.first; });
        size_t w = 0;
        for (size_t k2 = 0; k2 < r.size(); ++k2) {
            if (w > 0 && r[w - 1].first == r[k2].first) r[w - 1].second += r[k2].second;
            else r[w++] = r[k2];
        }
        r.resize(w);
        for (auto &kv : r) { M.m_ci.push_back(M.free_edges[kv.first]); M.m_v.push_back(kv.second); }
        M.m_rp[i + 1] = (long long)M.m_ci.size();
    }
    return FETDPIC_OK;
}

}  // namespace fetdpic
