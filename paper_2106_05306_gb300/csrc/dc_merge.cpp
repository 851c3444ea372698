// Packing several cloth instances into one context: their meshes, prefactored
// PD matrices and adjoint front structures are concatenated into one
// disconnected problem.  P is then block diagonal, every per-element and per-row
// kernel covers all instances in one launch, and no value of one instance
// depends on another (the factor, the explicit inverse rows and the fronts of
// each instance are exactly those it has alone).
#include <algorithm>

#include "dc_internal.h"

void dc_merge_meshes(const std::vector<HostMesh>& H, std::vector<InstInfo>& I, HostMesh& out) {
    const int B = (int)H.size();
    I.assign(B, InstInfo());
    int MF = 0, M = 0, T = 0, pins = 0;
    long long ext = 0;
    for (int i = 0; i < B; ++i) {
        I[i].m = H[i].m;
        I[i].mf = H[i].m_free;
        I[i].T = H[i].T;
        I[i].ext_off = ext;
        I[i].fo = MF;
        I[i].po = pins;
        I[i].to = T;
        ext += H[i].m;
        MF += H[i].m_free;
        pins += H[i].m - H[i].m_free;
        M += H[i].m;
        T += H[i].T;
    }
    out = HostMesh();
    out.m = M;
    out.m_free = MF;
    out.T = T;
    out.int2ext.assign(M, 0);
    out.ext2int.assign(M, 0);
    out.rest.assign(3 * (size_t)M, 0.0);
    out.abar.assign(M, 0.0);
    out.sb.assign(M, 0.0);
    out.qrest.assign(3 * (size_t)M, 0.0);
    out.tri.reserve(3 * (size_t)T);
    out.G.reserve(4 * (size_t)T);
    out.area.reserve(T);
    for (int i = 0; i < B; ++i) {
        const HostMesh& h = H[i];
        out.nd_depth = std::max(out.nd_depth, h.nd_depth);
        for (int l = 0; l < h.m; ++l) {
            const int g = I[i].map(l, MF);
            out.int2ext[g] = (int)(I[i].ext_off + h.int2ext[l]);
            out.ext2int[out.int2ext[g]] = g;
            for (int k = 0; k < 3; ++k) {
                out.rest[3 * (size_t)g + k] = h.rest[3 * (size_t)l + k];
                out.qrest[3 * (size_t)g + k] = h.qrest[3 * (size_t)l + k];
            }
            out.abar[g] = h.abar[l];
            out.sb[g] = h.sb[l];
        }
        for (int t = 0; t < h.T; ++t) {
            for (int a = 0; a < 3; ++a) out.tri.push_back(I[i].map(h.tri[3 * t + a], MF));
            for (int k = 0; k < 4; ++k) out.G.push_back(h.G[4 * (size_t)t + k]);
            out.area.push_back(h.area[t]);
        }
    }
    // bending rows in merged node order: free nodes of every instance, then pins
    out.bptr.assign(1, 0);
    auto add_row = [&](int i, int l) {
        const HostMesh& h = H[i];
        for (int k = h.bptr[l]; k < h.bptr[l + 1]; ++k) {
            out.bidx.push_back(I[i].map(h.bidx[k], MF));
            out.bval.push_back(h.bval[k]);
        }
        out.bptr.push_back((int)out.bidx.size());
    };
    for (int i = 0; i < B; ++i)
        for (int l = 0; l < H[i].m_free; ++l) add_row(i, l);
    for (int i = 0; i < B; ++i)
        for (int l = H[i].m_free; l < H[i].m; ++l) add_row(i, l);
}

void dc_merge_factors(const std::vector<HostFactor>& F, const std::vector<InstInfo>& I, HostFactor& out) {
    out = HostFactor();
    out.fptr.assign(1, 0);
    out.bptr.assign(1, 0);
    long long nnz = 0;
    for (size_t i = 0; i < F.size(); ++i) {
        const HostFactor& f = F[i];
        const int fo = I[i].fo;
        out.n += f.n;
        nnz += f.colptr.empty() ? 0 : f.colptr.back();
        for (int r = 0; r < f.n; ++r) {
            for (int k = f.fptr[r]; k < f.fptr[r + 1]; ++k) {
                out.fidx.push_back(f.fidx[k] + fo);
                out.fval.push_back(f.fval[k]);
            }
            out.fptr.push_back((int)out.fidx.size());
            for (int k = f.bptr[r]; k < f.bptr[r + 1]; ++k) {
                out.bidx.push_back(f.bidx[k] + fo);
                out.bval.push_back(f.bval[k]);
            }
            out.bptr.push_back((int)out.bidx.size());
        }
        out.max_diag = std::max(out.max_diag, f.max_diag);
    }
    // only the size of the scalar factor is kept (statistics)
    out.colptr.assign(1, (int)std::min<long long>(nnz, 0x7fffffff));
}

void dc_merge_fronts(const std::vector<HostFronts>& F, std::vector<InstInfo>& I, int MF, HostFronts& out) {
    out = HostFronts();
    out.uptr.assign(1, 0);
    out.cptr.assign(1, 0);
    out.pr_cptr.assign(1, 0);
    long long pool = 0, acc = 0, binv = 0, linv = 0;
    int nlev = 0;
    for (size_t i = 0; i < F.size(); ++i) {
        const HostFronts& f = F[i];
        InstInfo& in = I[i];
        in.so = out.S;
        const int so = out.S, fo = in.fo, to = in.to;
        for (int s = 0; s < f.S; ++s) {
            out.begin.push_back(f.begin[s] + fo);
            out.end.push_back(f.end[s] + fo);
            out.parent.push_back(f.parent[s] >= 0 ? f.parent[s] + so : -1);
            out.level.push_back(f.level[s]);
            out.f.push_back(f.f[s]);
            out.p.push_back(f.p[s]);
            out.off.push_back(f.off[s] + pool);
            out.acc_off.push_back(f.acc_off[s] + acc);
            out.binv_off.push_back(f.binv_off[s] + binv);
            out.linv_off.push_back(f.linv_off[s] + linv);
            for (int k = f.uptr[s]; k < f.uptr[s + 1]; ++k) {
                out.unode.push_back(f.unode[k] + fo);
                out.cmap.push_back(f.cmap[k]);
            }
            out.uptr.push_back((int)out.unode.size());
            for (int k = f.cptr[s]; k < f.cptr[s + 1]; ++k) out.child.push_back(f.child[k] + so);
            out.cptr.push_back((int)out.child.size());
            nlev = std::max(nlev, f.level[s] + 1);
        }
        for (size_t q = 0; q < f.pr_i.size(); ++q) {
            out.pr_i.push_back(f.pr_i[q] + fo);
            out.pr_j.push_back(f.pr_j[q] + fo);
            out.pr_ld.push_back(f.pr_ld[q]);
            out.pr_dst.push_back(f.pr_dst[q] + pool);
            for (int k = f.pr_cptr[q]; k < f.pr_cptr[q + 1]; ++k) {
                const int code = f.pr_code[k];
                // triangle codes t*9 + a*3 + b; bending codes -(b + 1) with b a node
                out.pr_code.push_back(code >= 0 ? code + 9 * to : -(in.map(-code - 1, MF) + 1));
                out.pr_coef.push_back(f.pr_coef[k]);
            }
            out.pr_cptr.push_back((int)out.pr_code.size());
        }
        out.S += f.S;
        out.max_f = std::max(out.max_f, f.max_f);
        pool += f.pool_size;
        acc += f.acc_size;
        binv += f.binv_size;
        linv += f.linv_size;
    }
    out.pool_size = pool;
    out.acc_size = acc;
    out.binv_size = binv;
    out.linv_size = linv;
    // levels by height (leaves 0): a front's children all have a smaller height
    out.lvl_ptr.assign(nlev + 1, 0);
    for (int s = 0; s < out.S; ++s) out.lvl_ptr[out.level[s] + 1]++;
    for (int l = 0; l < nlev; ++l) out.lvl_ptr[l + 1] += out.lvl_ptr[l];
    out.lvl_sn.assign(out.S, 0);
    std::vector<int> fill(out.lvl_ptr.begin(), out.lvl_ptr.end() - 1);
    for (int s = 0; s < out.S; ++s) out.lvl_sn[fill[out.level[s]]++] = s;
}
