// Host-side symbolic structure of the per-step multifrontal LDL^T that the
// adjoint uses as its preconditioner (the matrix H of Sec. 4, Eq. ppr_adjoint,
// with the contact constraints applied per node).
//
// H has the node-level sparsity of P (every element couples the same nodes), so
// the elimination tree and column structures of P's Cholesky factor apply.
// Supernodes are maximal runs of consecutive columns j, j+1 with
// parent(j) = j+1 inside one nested-dissection block; the front of supernode s
// holds its own nodes followed by U_s = struct(last column of s).  Fronts are
// processed level by level (leaves first); each child's update block is added
// into its parent's front through a node-position map.
#include <algorithm>
#include <string>
#include <vector>

#include "dc_internal.h"

std::string dc_build_fronts(const HostMesh& hm, const HostFactor& hf, HostFronts& fr) {
    const int n = hf.n;
    fr = HostFronts();
    // ---- supernodes
    std::vector<int> sn_of(n, -1);
    for (int j = 0; j < n; ++j) {
        bool cont = j > 0 && hm.nd_block[j] == hm.nd_block[j - 1] && hf.parent[j - 1] == j;
        if (!cont) {
            fr.begin.push_back(j);
            fr.end.push_back(j + 1);
        } else {
            fr.end.back() = j + 1;
        }
        sn_of[j] = (int)fr.begin.size() - 1;
    }
    const int S = (int)fr.begin.size();
    fr.S = S;
    fr.parent.assign(S, -1);
    fr.uptr.assign(1, 0);
    for (int s = 0; s < S; ++s) {
        int last = fr.end[s] - 1;
        for (int q = hf.colptr[last] + 1; q < hf.colptr[last + 1]; ++q) fr.unode.push_back(hf.rowidx[q]);
        fr.uptr.push_back((int)fr.unode.size());
        int par = hf.parent[last];
        fr.parent[s] = par >= 0 ? sn_of[par] : -1;
        if (fr.parent[s] >= 0 && fr.parent[s] <= s) return "supernode tree is not in post-order";
    }
    // children lists
    std::vector<std::vector<int>> ch(S);
    for (int s = 0; s < S; ++s)
        if (fr.parent[s] >= 0) ch[fr.parent[s]].push_back(s);
    fr.cptr.assign(1, 0);
    for (int s = 0; s < S; ++s) {
        for (int c : ch[s]) fr.child.push_back(c);
        fr.cptr.push_back((int)fr.child.size());
    }
    // sizes, offsets, levels
    fr.f.resize(S);
    fr.p.resize(S);
    fr.off.resize(S);
    fr.acc_off.resize(S);
    fr.binv_off.resize(S);
    fr.linv_off.resize(S);
    fr.level.assign(S, 0);
    long long off = 0, acc = 0, binv = 0, linv = 0;
    fr.max_f = 0;
    for (int s = 0; s < S; ++s) {
        int ns = fr.end[s] - fr.begin[s];
        int nu = fr.uptr[s + 1] - fr.uptr[s];
        fr.p[s] = 3 * ns;
        fr.f[s] = 3 * (ns + nu);
        fr.max_f = std::max(fr.max_f, fr.f[s]);
        fr.off[s] = off;
        off += ((long long)fr.f[s] * fr.f[s] + 31) / 32 * 32;
        fr.acc_off[s] = acc;
        acc += (3LL * nu + 31) / 32 * 32;
        fr.binv_off[s] = binv;
        binv += (long long)((fr.p[s] + 31) / 32) * 32 * 32;
        fr.linv_off[s] = linv;
        linv += ((long long)fr.p[s] * fr.p[s] + 31) / 32 * 32;
        for (int c : ch[s]) fr.level[s] = std::max(fr.level[s], fr.level[c] + 1);
    }
    fr.pool_size = off;
    fr.acc_size = acc;
    fr.binv_size = binv;
    fr.linv_size = linv;
    int nlev = 0;
    for (int s = 0; s < S; ++s) nlev = std::max(nlev, fr.level[s] + 1);
    fr.lvl_ptr.assign(nlev + 1, 0);
    for (int s = 0; s < S; ++s) fr.lvl_ptr[fr.level[s] + 1]++;
    for (int l = 0; l < nlev; ++l) fr.lvl_ptr[l + 1] += fr.lvl_ptr[l];
    fr.lvl_sn.assign(S, 0);
    {
        std::vector<int> fill(fr.lvl_ptr.begin(), fr.lvl_ptr.end() - 1);
        for (int s = 0; s < S; ++s) fr.lvl_sn[fill[fr.level[s]]++] = s;
    }
    // child -> parent position maps: position of U_c[k] in the parent's node list
    fr.cmap.assign(fr.unode.size(), -1);
    for (int c = 0; c < S; ++c) {
        int par = fr.parent[c];
        if (par < 0) {
            if (fr.uptr[c + 1] != fr.uptr[c]) return "root supernode with a non-empty update";
            continue;
        }
        const int* pu = fr.unode.data() + fr.uptr[par];
        int npu = fr.uptr[par + 1] - fr.uptr[par];
        for (int k = fr.uptr[c]; k < fr.uptr[c + 1]; ++k) {
            int node = fr.unode[k];
            int pos;
            if (node >= fr.begin[par] && node < fr.end[par]) {
                pos = node - fr.begin[par];
            } else {
                const int* it = std::lower_bound(pu, pu + npu, node);
                if (it == pu + npu || *it != node) return "update row missing from the parent front";
                pos = (fr.end[par] - fr.begin[par]) + (int)(it - pu);
            }
            fr.cmap[k] = pos;
        }
    }
    // ---- node pairs (i >= j, both free) of H's lower pattern and their contributions
    std::vector<std::vector<int>> rows(n);
    auto add_pair = [&](int i, int j) {
        if (i < j) std::swap(i, j);
        if (i < n && j < n) rows[j].push_back(i);
    };
    for (int j = 0; j < n; ++j) add_pair(j, j);
    for (int t = 0; t < hm.T; ++t)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) add_pair(hm.tri[3 * t + a], hm.tri[3 * t + b]);
    for (int b = 0; b < hm.m; ++b)
        for (int u = hm.bptr[b]; u < hm.bptr[b + 1]; ++u)
            for (int v = hm.bptr[b]; v < hm.bptr[b + 1]; ++v) add_pair(hm.bidx[u], hm.bidx[v]);
    std::vector<int> colstart(n + 1, 0);
    for (int j = 0; j < n; ++j) {
        std::sort(rows[j].begin(), rows[j].end());
        rows[j].erase(std::unique(rows[j].begin(), rows[j].end()), rows[j].end());
        colstart[j + 1] = colstart[j] + (int)rows[j].size();
    }
    const int NP = colstart[n];
    fr.pr_i.resize(NP);
    fr.pr_j.resize(NP);
    fr.pr_dst.resize(NP);
    fr.pr_ld.resize(NP);
    for (int j = 0; j < n; ++j) {
        int s = sn_of[j];
        const int* pu = fr.unode.data() + fr.uptr[s];
        int npu = fr.uptr[s + 1] - fr.uptr[s];
        int ns = fr.end[s] - fr.begin[s];
        int pj = j - fr.begin[s];
        for (int q = 0; q < (int)rows[j].size(); ++q) {
            int i = rows[j][q];
            int pi;
            if (i < fr.end[s]) {
                pi = i - fr.begin[s];
            } else {
                const int* it = std::lower_bound(pu, pu + npu, i);
                if (it == pu + npu || *it != i) return "matrix entry outside its front";
                pi = ns + (int)(it - pu);
            }
            int id = colstart[j] + q;
            fr.pr_i[id] = i;
            fr.pr_j[id] = j;
            fr.pr_ld[id] = fr.f[s];
            fr.pr_dst[id] = fr.off[s] + (long long)(3 * pj) * fr.f[s] + 3 * pi;
        }
    }
    auto pair_id = [&](int i, int j) {
        const std::vector<int>& r = rows[j];
        return colstart[j] + (int)(std::lower_bound(r.begin(), r.end(), i) - r.begin());
    };
    std::vector<std::vector<std::pair<int, double>>> contrib(NP);
    for (int t = 0; t < hm.T; ++t)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int i = hm.tri[3 * t + a], j = hm.tri[3 * t + b];
                if (i < j || i >= n || j >= n) continue;
                contrib[pair_id(i, j)].push_back({t * 9 + a * 3 + b, 0.0});
            }
    for (int b = 0; b < hm.m; ++b)
        for (int u = hm.bptr[b]; u < hm.bptr[b + 1]; ++u)
            for (int v = hm.bptr[b]; v < hm.bptr[b + 1]; ++v) {
                int i = hm.bidx[u], j = hm.bidx[v];
                if (i < j || i >= n || j >= n) continue;
                contrib[pair_id(i, j)].push_back({-(b + 1), hm.bval[u] * hm.bval[v]});
            }
    fr.pr_cptr.assign(1, 0);
    for (int id = 0; id < NP; ++id) {
        for (auto& e : contrib[id]) {
            fr.pr_code.push_back(e.first);
            fr.pr_coef.push_back(e.second);
        }
        fr.pr_cptr.push_back((int)fr.pr_code.size());
    }
    return "";
}

void dc_build_psolve(const HostFactor& hf, const HostFronts& fr, HostPSolve& ps, bool values) {
    const int S = fr.S;
    ps = HostPSolve();
    ps.poff.resize(S);
    ps.xoff.resize(S);
    ps.toff.resize(S);
    ps.aoff.resize(S);
    long long po = 0, xo = 0, to = 0, ao = 0;
    for (int s = 0; s < S; ++s) {
        const long long ns = fr.end[s] - fr.begin[s], nu = fr.uptr[s + 1] - fr.uptr[s];
        ps.poff[s] = po;
        ps.xoff[s] = xo;
        ps.toff[s] = to;
        ps.aoff[s] = (int)ao;
        po += (ns + nu) * ns;
        xo += ns * ns;
        to += ns * nu;
        ao += nu;
    }
    ps.acc_nodes = ao;
    ps.n_panel = po;
    ps.n_xinv = xo;
    ps.n_pant = to;
    if (!values) return;
    ps.panel.assign(po, 0.0);
    ps.xinv.assign(xo, 0.0);
    ps.xinvt.assign(xo, 0.0);
    ps.pant.assign(to, 0.0);
    std::vector<double> x;
    for (int s = 0; s < S; ++s) {
        const int b = fr.begin[s], e = fr.end[s], ns = e - b;
        const int* un = fr.unode.data() + fr.uptr[s];
        const int nu = fr.uptr[s + 1] - fr.uptr[s], fs = ns + nu;
        double* pan = ps.panel.data() + ps.poff[s];
        for (int c = 0; c < ns; ++c) {
            const int j = b + c;
            for (int q = hf.colptr[j]; q < hf.colptr[j + 1]; ++q) {
                const int i = hf.rowidx[q];
                const int pos = i < e ? i - b : ns + (int)(std::lower_bound(un, un + nu, i) - un);
                pan[(long)c * fs + pos] = hf.val[q];
            }
        }
        // inverse of the top block D (D[r][c] = pan[c * fs + r], lower) column by column
        double* X = ps.xinv.data() + ps.xoff[s];
        x.assign(ns, 0.0);
        for (int c = 0; c < ns; ++c) {
            for (int r = 0; r < ns; ++r) x[r] = 0.0;
            for (int r = c; r < ns; ++r) {
                double t = (r == c) ? 1.0 : 0.0;
                for (int k = c; k < r; ++k) t -= pan[(long)k * fs + r] * x[k];
                x[r] = t / pan[(long)r * fs + r];
            }
            for (int r = 0; r < ns; ++r) X[(long)c * ns + r] = x[r];
        }
        // transposed copies for the backward sweep
        double* XT = ps.xinvt.data() + ps.xoff[s];
        for (int c = 0; c < ns; ++c)
            for (int r = 0; r < ns; ++r) XT[(long)r * ns + c] = X[(long)c * ns + r];
        double* T = ps.pant.data() + ps.toff[s];
        for (int c = 0; c < ns; ++c)
            for (int k = 0; k < nu; ++k) T[(long)k * ns + c] = pan[(long)c * fs + ns + k];
    }
}

void dc_merge_psolve(const std::vector<HostPSolve>& P, HostPSolve& out) {
    out = HostPSolve();
    long long po = 0, xo = 0, to = 0, ao = 0;
    for (const HostPSolve& p : P) {
        for (size_t s = 0; s < p.poff.size(); ++s) {
            out.poff.push_back(p.poff[s] + po);
            out.xoff.push_back(p.xoff[s] + xo);
            out.toff.push_back(p.toff[s] + to);
            out.aoff.push_back((int)(p.aoff[s] + ao));
        }
        out.panel.insert(out.panel.end(), p.panel.begin(), p.panel.end());
        out.xinv.insert(out.xinv.end(), p.xinv.begin(), p.xinv.end());
        out.xinvt.insert(out.xinvt.end(), p.xinvt.begin(), p.xinvt.end());
        out.pant.insert(out.pant.end(), p.pant.begin(), p.pant.end());
        po += p.n_panel;
        xo += p.n_xinv;
        to += p.n_pant;
        ao += p.acc_nodes;
    }
    out.acc_nodes = ao;
    out.n_panel = po;
    out.n_xinv = xo;
    out.n_pant = to;
}

// Work items of the tree-scheduled sweeps, in a topological order (every front
// after its children): fronts farther from their root come first, so the longest
// remaining chains start earliest.  A front of more than DC_PS_SMALL nodes is an
// item alone (one CTA); smaller fronts of equal depth go up to DC_PS_WARPS to an
// item (one warp each).  Item q is tq_sn[tq_ptr[q] .. tq_ptr[q + 1]).
void dc_build_tree_items(const HostFronts& fr, std::vector<int>& tq_ptr, std::vector<int>& tq_sn) {
    std::vector<int> depth(fr.S, 0), order(fr.S);
    for (int s = 0; s < fr.S; ++s) {
        order[s] = s;
        for (int a = fr.parent[s]; a >= 0; a = fr.parent[a]) depth[s]++;
    }
    auto large = [&](int s) { return fr.f[s] / 3 > DC_PS_SMALL; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (depth[a] != depth[b]) return depth[a] > depth[b];
        return large(a) && !large(b);
    });
    tq_ptr.assign(1, 0);
    tq_sn.clear();
    for (size_t k = 0; k < order.size();) {
        const int s = order[k];
        if (large(s)) {
            tq_sn.push_back(s);
            ++k;
        } else {
            for (int n = 0; k < order.size() && n < DC_PS_WARPS && !large(order[k]) && depth[order[k]] == depth[s]; ++n)
                tq_sn.push_back(order[k++]);
        }
        tq_ptr.push_back((int)tq_sn.size());
    }
}

// For every front s and node position t of s (t < f_s / 3, pivots first): the
// update-vector entries of s's children that add into t, children in cptr order
// and entries in ascending order (entry j of child c is aoff[c] + stride j), so that a gather summing them in list order
// adds exactly what a child-by-child scatter adds.
void dc_build_pull_lists(const HostFronts& fr, const std::vector<int>& aoff, int stride, std::vector<int>& pull_off,
                         std::vector<int>& pull_ptr, std::vector<int>& pull_idx) {
    pull_off.assign(fr.S, 0);
    pull_ptr.clear();
    pull_idx.clear();
    std::vector<int> fill;
    for (int s = 0; s < fr.S; ++s) {
        const int fs = fr.f[s] / 3;
        pull_off[s] = (int)pull_ptr.size();
        const size_t base = pull_ptr.size();
        pull_ptr.resize(base + fs + 1, 0);
        for (int q = fr.cptr[s]; q < fr.cptr[s + 1]; ++q) {
            const int c = fr.child[q];
            for (int k = fr.uptr[c]; k < fr.uptr[c + 1]; ++k) pull_ptr[base + fr.cmap[k] + 1]++;
        }
        pull_ptr[base] = (int)pull_idx.size();
        for (int t = 0; t < fs; ++t) pull_ptr[base + t + 1] += pull_ptr[base + t];
        pull_idx.resize(pull_ptr[base + fs]);
        fill.assign(pull_ptr.begin() + base, pull_ptr.begin() + base + fs);
        for (int q = fr.cptr[s]; q < fr.cptr[s + 1]; ++q) {
            const int c = fr.child[q];
            for (int k = fr.uptr[c]; k < fr.uptr[c + 1]; ++k)
                pull_idx[fill[fr.cmap[k]]++] = aoff[c] + stride * (k - fr.uptr[c]);
        }
    }
}
