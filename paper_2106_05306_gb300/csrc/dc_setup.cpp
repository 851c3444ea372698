// Host-side, once-per-mesh and once-per-parameter-set work of libdc:
//  * rest-shape operators of the PD energies (Sec. 3.1, Eq. pd_project, with the
//    triangle-stretch and vertex-bending readings of the cloth model the paper
//    cites: per-triangle G = E Dm^-1 and rest area; per-vertex cotangent
//    Laplacian row over the vertex area; lumped mass);
//  * a nested-dissection ordering of the free nodes (recursive coordinate
//    bisection with vertex separators taken from the graph of P);
//  * assembly of P = M + h^2 sum_i w_i A_i^T A_i (Eq. pd_global) on free nodes
//    and its sparse Cholesky factor P = L L^T (elimination tree, symbolic
//    column structures, left-looking numeric factorisation);
//  * the explicit inverse factor L^-1 (rows for the forward substitution, and
//    its transpose for the backward substitution) used by the GPU solve.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "dc_internal.h"

namespace {

struct V3 {
    double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 scale(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }

// Recursive coordinate bisection.  Appends the nodes of `nodes` to `order`
// (sub-domains first, separator last) and records each node's tree depth.
void nd_recurse(const std::vector<std::vector<int>>& adj, const std::vector<double>& xyz,
                std::vector<int> nodes, std::vector<int>& order, std::vector<int>& level,
                std::vector<int>& side, int depth, int& maxdepth, size_t leaf, std::vector<int>& block,
                int& nblock) {
    maxdepth = std::max(maxdepth, depth);
    if (nodes.size() <= leaf) {
        std::sort(nodes.begin(), nodes.end());
        int id = nblock++;
        for (int u : nodes) {
            order.push_back(u);
            level[u] = depth;
            block[u] = id;
        }
        return;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int u : nodes)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], xyz[3 * u + c]);
            hi[c] = std::max(hi[c], xyz[3 * u + c]);
        }
    int ax = 0;
    for (int c = 1; c < 3; ++c)
        if (hi[c] - lo[c] > hi[ax] - lo[ax]) ax = c;
    std::sort(nodes.begin(), nodes.end(), [&](int a, int b) {
        double ca = xyz[3 * a + ax], cb = xyz[3 * b + ax];
        return ca < cb || (ca == cb && a < b);
    });
    size_t half = nodes.size() / 2;
    // keep nodes with equal coordinate on the same side
    double cut = xyz[3 * nodes[half] + ax];
    size_t nl = 0;
    while (nl < nodes.size() && xyz[3 * nodes[nl] + ax] < cut) ++nl;
    if (nl == 0 || nl == nodes.size()) nl = half;
    for (size_t i = 0; i < nodes.size(); ++i) side[nodes[i]] = (i < nl) ? 1 : 2;
    std::vector<int> L, R, S;
    for (size_t i = 0; i < nl; ++i) {
        int u = nodes[i];
        bool touches = false;
        for (int v : adj[u])
            if (side[v] == 2) {
                touches = true;
                break;
            }
        (touches ? S : L).push_back(u);
    }
    for (size_t i = nl; i < nodes.size(); ++i) R.push_back(nodes[i]);
    for (int u : nodes) side[u] = 0;
    if (L.empty() && R.empty()) {
        int id = nblock++;
        for (int u : S) {
            order.push_back(u);
            level[u] = depth;
            block[u] = id;
        }
        return;
    }
    if (!L.empty()) nd_recurse(adj, xyz, L, order, level, side, depth + 1, maxdepth, leaf, block, nblock);
    if (!R.empty()) nd_recurse(adj, xyz, R, order, level, side, depth + 1, maxdepth, leaf, block, nblock);
    std::sort(S.begin(), S.end());
    int id = nblock++;
    for (int u : S) {
        order.push_back(u);
        level[u] = depth;
        block[u] = id;
    }
}

}  // namespace

std::string dc_build_mesh(HostMesh& hm, int m, const double* rest_pos, int T, const int32_t* tris,
                          int n_pins, const int32_t* pins) {
    if (m < 3 || T < 1) return "mesh needs at least 3 nodes and 1 triangle";
    for (int i = 0; i < 3 * m; ++i)
        if (!std::isfinite(rest_pos[i])) return "non-finite rest position";
    for (int i = 0; i < 3 * T; ++i)
        if (tris[i] < 0 || tris[i] >= m) return "triangle index out of range";
    std::vector<char> is_pin(m, 0);
    for (int i = 0; i < n_pins; ++i) {
        if (pins[i] < 0 || pins[i] >= m) return "pin index out of range";
        is_pin[pins[i]] = 1;
    }
    hm.m = m;
    hm.T = T;

    // ---- triangles, external numbering first (Dm, G, area)
    std::vector<double> G(4 * (size_t)T), area(T);
    auto P3 = [&](int i) { return V3{rest_pos[3 * i], rest_pos[3 * i + 1], rest_pos[3 * i + 2]}; };
    for (int t = 0; t < T; ++t) {
        int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        if (a == b || b == c || a == c) return "degenerate triangle (repeated node)";
        V3 e1 = sub(P3(b), P3(a)), e2 = sub(P3(c), P3(a));
        V3 cr = cross(e1, e2);
        double l1 = norm(e1), lc = norm(cr);
        if (!(l1 > 0) || !(lc > 0)) return "triangle with zero rest area";
        area[t] = 0.5 * lc;
        V3 u = scale(e1, 1.0 / l1);
        V3 nrm = scale(cr, 1.0 / lc);
        V3 w = cross(nrm, u);
        // Dm = [[e1.u, e2.u], [e1.w, e2.w]] (e1.w = 0 up to rounding)
        double d00 = dot(e1, u), d01 = dot(e2, u), d10 = dot(e1, w), d11 = dot(e2, w);
        double det = d00 * d11 - d01 * d10;
        // G = E Dm^-1: row 1 = first row of Dm^-1, row 2 = second row
        G[4 * t + 0] = d11 / det;
        G[4 * t + 1] = -d01 / det;
        G[4 * t + 2] = -d10 / det;
        G[4 * t + 3] = d00 / det;
    }

    // ---- cotangent weights c_ij = (cot a + cot b)/2 and vertex areas
    std::vector<std::map<int, double>> W(m);
    std::vector<double> abar(m, 0.0);
    for (int t = 0; t < T; ++t) {
        for (int k = 0; k < 3; ++k) {
            int o = tris[3 * t + k], i = tris[3 * t + (k + 1) % 3], j = tris[3 * t + (k + 2) % 3];
            V3 a = sub(P3(i), P3(o)), b = sub(P3(j), P3(o));
            double cot = dot(a, b) / norm(cross(a, b));
            W[i][j] += 0.5 * cot;
            W[j][i] += 0.5 * cot;
            abar[tris[3 * t + k]] += area[t] / 3.0;
        }
    }

    // ---- adjacency of P's sparsity (triangle edges + pairs inside a bending stencil)
    std::vector<std::vector<int>> adjx(m);
    auto link = [&](int a, int b) {
        if (a != b) {
            adjx[a].push_back(b);
            adjx[b].push_back(a);
        }
    };
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) link(tris[3 * t + k], tris[3 * t + (k + 1) % 3]);
    for (int b = 0; b < m; ++b) {
        std::vector<int> st{b};
        for (auto& kv : W[b]) st.push_back(kv.first);
        for (size_t p = 0; p < st.size(); ++p)
            for (size_t q = p + 1; q < st.size(); ++q) link(st[p], st[q]);
    }
    for (auto& a : adjx) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }

    // ---- nested dissection on free nodes
    std::vector<int> freen;
    for (int i = 0; i < m; ++i)
        if (!is_pin[i]) freen.push_back(i);
    if (freen.empty()) return "every node is pinned";
    std::vector<std::vector<int>> adjf(m);
    for (int u : freen)
        for (int v : adjx[u])
            if (!is_pin[v]) adjf[u].push_back(v);
    std::vector<double> xyz(rest_pos, rest_pos + 3 * (size_t)m);
    std::vector<int> order, lvl(m, 0), side(m, 0), blk(m, -1);
    int maxdepth = 0, nblock = 0;
    nd_recurse(adjf, xyz, freen, order, lvl, side, 0, maxdepth, 24, blk, nblock);
    hm.m_free = (int)order.size();
    for (int i = 0; i < m; ++i)
        if (is_pin[i]) order.push_back(i);
    hm.int2ext = order;
    hm.ext2int.assign(m, -1);
    for (int i = 0; i < m; ++i) hm.ext2int[order[i]] = i;
    hm.nd_depth = maxdepth;
    hm.nd_level.resize(hm.m_free);
    hm.nd_block.resize(hm.m_free);
    for (int i = 0; i < hm.m_free; ++i) {
        hm.nd_level[i] = lvl[order[i]];
        hm.nd_block[i] = blk[order[i]];
    }

    // ---- store everything in internal numbering
    hm.rest.resize(3 * (size_t)m);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < 3; ++c) hm.rest[3 * i + c] = rest_pos[3 * order[i] + c];
    hm.tri.resize(3 * (size_t)T);
    for (int i = 0; i < 3 * T; ++i) hm.tri[i] = hm.ext2int[tris[i]];
    hm.G = G;
    hm.area = area;
    hm.abar.resize(m);
    for (int i = 0; i < m; ++i) hm.abar[i] = abar[order[i]];

    // bending rows l_b (internal), q_rest = A_b x_rest, s_b = |q_rest| (0 where flat)
    double cx = 0, cy = 0, cz = 0;
    for (int i = 0; i < m; ++i) {
        cx += rest_pos[3 * i];
        cy += rest_pos[3 * i + 1];
        cz += rest_pos[3 * i + 2];
    }
    cx /= m;
    cy /= m;
    cz /= m;
    double rad = 0;
    for (int i = 0; i < m; ++i)
        rad = std::max(rad, norm(V3{rest_pos[3 * i] - cx, rest_pos[3 * i + 1] - cy, rest_pos[3 * i + 2] - cz}));
    hm.bptr.assign(1, 0);
    hm.bidx.clear();
    hm.bval.clear();
    hm.sb.assign(m, 0.0);
    hm.qrest.assign(3 * (size_t)m, 0.0);
    for (int bi = 0; bi < m; ++bi) {
        int b = order[bi];
        double inv_a = 1.0 / abar[b];
        double deg = 0, absum = 0;
        std::vector<std::pair<int, double>> row;
        for (auto& kv : W[b]) {
            deg += kv.second;
            row.push_back({hm.ext2int[kv.first], kv.second * inv_a});
        }
        row.push_back({bi, -deg * inv_a});
        std::sort(row.begin(), row.end());
        V3 q{0, 0, 0};
        for (auto& e : row) {
            hm.bidx.push_back(e.first);
            hm.bval.push_back(e.second);
            absum += std::fabs(e.second);
            int ex = order[e.first];
            q.x += e.second * rest_pos[3 * ex];
            q.y += e.second * rest_pos[3 * ex + 1];
            q.z += e.second * rest_pos[3 * ex + 2];
        }
        hm.bptr.push_back((int)hm.bidx.size());
        double s = norm(q);
        hm.sb[bi] = (s <= 1e-9 * absum * rad) ? 0.0 : s;
        hm.qrest[3 * bi] = q.x;
        hm.qrest[3 * bi + 1] = q.y;
        hm.qrest[3 * bi + 2] = q.z;
    }
    return "";
}

dc_status dc_build_factor(const HostMesh& hm, const dc_params& p, const std::vector<double>& mass,
                          HostFactor& hf, std::string& err, bool symbolic_only) {
    const int n = hm.m_free;
    const double h2 = p.h * p.h;
    // ---- assemble the lower triangle of P_ff by columns (map per column)
    std::vector<std::map<int, double>> col(n);
    auto add = [&](int i, int j, double v) {   // internal indices; keep i >= j, both free
        if (i >= n || j >= n) return;
        if (i < j) std::swap(i, j);
        col[j][i] += v;
    };
    for (int i = 0; i < n; ++i) add(i, i, mass[i]);
    hf.max_diag = 0.0;
    for (int t = 0; t < hm.T; ++t) {
        const double* g = &hm.G[4 * t];
        double gr[3][2] = {{-(g[0] + g[2]), -(g[1] + g[3])}, {g[0], g[1]}, {g[2], g[3]}};
        double w = p.k_stretch * hm.area[t] * h2;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b <= a; ++b) {
                double v = w * (gr[a][0] * gr[b][0] + gr[a][1] * gr[b][1]);
                int ia = hm.tri[3 * t + a], ib = hm.tri[3 * t + b];
                if (a == b)
                    add(ia, ia, v);
                else
                    add(ia, ib, v);
            }
    }
    for (int b = 0; b < hm.m; ++b) {
        double w = p.k_bend * hm.abar[b] * h2;
        for (int u = hm.bptr[b]; u < hm.bptr[b + 1]; ++u)
            for (int v = hm.bptr[b]; v <= u; ++v) {
                double val = w * hm.bval[u] * hm.bval[v];
                int iu = hm.bidx[u], iv = hm.bidx[v];
                if (u == v)
                    add(iu, iu, val);
                else
                    add(iu, iv, val);
            }
    }
    hf.pdiag.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        hf.pdiag[j] = col[j][j];
        hf.max_diag = std::max(hf.max_diag, col[j][j]);
    }
    // ---- elimination tree (Liu's algorithm with path compression)
    std::vector<std::vector<int>> lower_rows(n);   // rows i > j of column j
    std::vector<std::vector<int>> upper_cols(n);   // for row i: columns j < i
    for (int j = 0; j < n; ++j)
        for (auto& kv : col[j])
            if (kv.first > j) {
                lower_rows[j].push_back(kv.first);
                upper_cols[kv.first].push_back(j);
            }
    std::vector<int> parent(n, -1), anc(n, -1);
    for (int i = 0; i < n; ++i)
        for (int j : upper_cols[i]) {
            int r = j;
            while (anc[r] != -1 && anc[r] != i) {
                int t = anc[r];
                anc[r] = i;
                r = t;
            }
            if (anc[r] == -1) {
                anc[r] = i;
                parent[r] = i;
            }
        }
    // ---- symbolic: struct(j) = rows(A(:,j) below j) U (struct(child) \ {j})
    std::vector<std::vector<int>> st(n);
    std::vector<std::vector<int>> children(n);
    for (int j = 0; j < n; ++j)
        if (parent[j] >= 0) children[parent[j]].push_back(j);
    for (int j = 0; j < n; ++j) {
        std::vector<int> s = lower_rows[j];
        for (int c : children[j])
            for (int r : st[c])
                if (r != j) s.push_back(r);
        std::sort(s.begin(), s.end());
        s.erase(std::unique(s.begin(), s.end()), s.end());
        st[j] = std::move(s);
    }
    // ---- CSC layout of L
    hf.n = n;
    hf.parent = parent;
    hf.colptr.assign(n + 1, 0);
    for (int j = 0; j < n; ++j) hf.colptr[j + 1] = hf.colptr[j] + 1 + (int)st[j].size();
    hf.rowidx.resize(hf.colptr[n]);
    hf.val.assign(hf.colptr[n], 0.0);
    for (int j = 0; j < n; ++j) {
        int q = hf.colptr[j];
        hf.rowidx[q++] = j;
        for (int r : st[j]) hf.rowidx[q++] = r;
    }
    if (symbolic_only) {
        hf.fptr.assign(n + 1, 0);
        hf.bptr.assign(n + 1, 0);
        hf.fidx.clear();
        hf.fval.clear();
        hf.bidx.clear();
        hf.bval.clear();
        return DC_OK;
    }
    // row access: for row i, the (column k, position of i in column k) with k < i
    std::vector<std::vector<std::pair<int, int>>> rowpos(n);
    for (int k = 0; k < n; ++k)
        for (int q = hf.colptr[k] + 1; q < hf.colptr[k + 1]; ++q) rowpos[hf.rowidx[q]].push_back({k, q});
    // ---- numeric, left-looking
    std::vector<double> x(n, 0.0);
    for (int j = 0; j < n; ++j) {
        for (auto& kv : col[j]) x[kv.first] = kv.second;
        for (auto& kq : rowpos[j]) {
            int k = kq.first;
            double ljk = hf.val[kq.second];
            for (int q = kq.second; q < hf.colptr[k + 1]; ++q) x[hf.rowidx[q]] -= hf.val[q] * ljk;
        }
        double d = x[j];
        if (!(d > 0.0) || !std::isfinite(d)) {
            err = "P is not positive definite (pivot " + std::to_string(d) + " at column " + std::to_string(j) + ")";
            return DC_ERR_NOT_SPD;
        }
        double ljj = std::sqrt(d);
        x[j] = 0.0;
        int q0 = hf.colptr[j];
        hf.val[q0] = ljj;
        for (int q = q0 + 1; q < hf.colptr[j + 1]; ++q) {
            hf.val[q] = x[hf.rowidx[q]] / ljj;
            x[hf.rowidx[q]] = 0.0;
        }
    }
    if (p.global_solver != 0) {   // the supernodal substitution uses L itself
        hf.fptr.assign(n + 1, 0);
        hf.bptr.assign(n + 1, 0);
        hf.fidx.clear();
        hf.fval.clear();
        hf.bidx.clear();
        hf.bval.clear();
        return DC_OK;
    }
    // ---- explicit inverse factor: column j of L^-1 lives on the etree path j -> root
    std::vector<std::vector<std::pair<int, double>>> inv_rows(n);   // row i: (col j, value)
    hf.bptr.assign(1, 0);
    hf.bidx.clear();
    hf.bval.clear();
    std::vector<int> path;
    for (int j = 0; j < n; ++j) {
        path.clear();
        for (int k = j; k != -1; k = parent[k]) path.push_back(k);
        x[j] = 1.0;
        for (int k : path) {
            double xk = x[k] / hf.val[hf.colptr[k]];
            x[k] = xk;
            for (int q = hf.colptr[k] + 1; q < hf.colptr[k + 1]; ++q) x[hf.rowidx[q]] -= hf.val[q] * xk;
        }
        // row j of L^-T = column j of L^-1 (rows ascending along the path)
        for (int k : path) {
            hf.bidx.push_back(k);
            hf.bval.push_back(x[k]);
            inv_rows[k].push_back({j, x[k]});
            x[k] = 0.0;
        }
        hf.bptr.push_back((int)hf.bidx.size());
    }
    hf.fptr.assign(1, 0);
    hf.fidx.clear();
    hf.fval.clear();
    for (int i = 0; i < n; ++i) {
        for (auto& e : inv_rows[i]) {      // columns ascending (j increases)
            hf.fidx.push_back(e.first);
            hf.fval.push_back(e.second);
        }
        hf.fptr.push_back((int)hf.fidx.size());
    }
    return DC_OK;
}

void dc_inverse_diagonal(const HostFactor& hf, std::vector<double>& zdiag) {
    const int n = hf.n;
    // Z on the pattern of L (same CSC positions); entries of column j depend only
    // on columns to its right, whose patterns contain every pair (i, k) of struct(j)
    std::vector<double> Z(hf.val.size(), 0.0);
    auto at = [&](int i, int k) -> double {   // Z_ik with i, k in struct of a common column
        if (i < k) std::swap(i, k);            // lower triangle: row i of column k
        const int* lo = hf.rowidx.data() + hf.colptr[k];
        const int* hi = hf.rowidx.data() + hf.colptr[k + 1];
        const int* p = std::lower_bound(lo, hi, i);
        return Z[p - hf.rowidx.data()];
    };
    for (int j = n - 1; j >= 0; --j) {
        const int q0 = hf.colptr[j], q1 = hf.colptr[j + 1];
        const double ljj = hf.val[q0];
        for (int a = q0 + 1; a < q1; ++a) {
            const int i = hf.rowidx[a];
            double s = 0.0;
            for (int b = q0 + 1; b < q1; ++b) s += hf.val[b] * at(i, hf.rowidx[b]);
            Z[a] = -s / ljj;
        }
        double s = 0.0;
        for (int b = q0 + 1; b < q1; ++b) s += hf.val[b] * Z[b];
        Z[q0] = 1.0 / (ljj * ljj) - s / ljj;
    }
    zdiag.assign(n, 0.0);
    for (int j = 0; j < n; ++j) zdiag[j] = Z[hf.colptr[j]];
}
