// Host-only check of the batch layout: builds three small grid cloths (different
// sizes, one with pins), factorises each, merges meshes, factors, fronts and
// supernodal panels as dc_create_batch / dc_set_params_batch do, and prints
// "ok" or the first broken invariant.  Compiled by tests/test_host_batch_layout.py
// from the library's host sources (no GPU needed).
#include <cstdio>
#include <set>
#include <string>
#include <vector>

#include "dc_internal.h"

static void grid(int n, std::vector<double>& pos, std::vector<int>& tri) {
    pos.clear();
    tri.clear();
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            pos.push_back(i / double(n - 1));
            pos.push_back(0.5);
            pos.push_back(j / double(n - 1));
        }
    for (int j = 0; j + 1 < n; ++j)
        for (int i = 0; i + 1 < n; ++i) {
            int a = j * n + i, b = a + 1, c = a + n, d = c + 1;
            tri.insert(tri.end(), {a, b, d, a, d, c});
        }
}

// The tree-scheduled sweeps' work items: every front in exactly one item, a
// large front alone, small fronts at most DC_PS_WARPS to an item and of one
// depth, and every child in an earlier item than its parent.  "" when valid.
static const char* check_items(const HostFronts& fr, int* n_large) {
    std::vector<int> tq_ptr, tq_sn;
    dc_build_tree_items(fr, tq_ptr, tq_sn);
    if ((int)tq_sn.size() != fr.S || tq_ptr.front() != 0 || tq_ptr.back() != fr.S) return "item sizes";
    std::vector<int> item(fr.S, -1), depth(fr.S, 0);
    for (int s = 0; s < fr.S; ++s)
        for (int a = fr.parent[s]; a >= 0; a = fr.parent[a]) depth[s]++;
    *n_large = 0;
    for (int q = 0; q + 1 < (int)tq_ptr.size(); ++q) {
        const int n = tq_ptr[q + 1] - tq_ptr[q];
        if (n < 1 || n > DC_PS_WARPS) return "item width";
        for (int k = tq_ptr[q]; k < tq_ptr[q + 1]; ++k) {
            const int s = tq_sn[k];
            if (s < 0 || s >= fr.S || item[s] >= 0) return "each front in one item";
            item[s] = q;
            const bool large = fr.f[s] / 3 > DC_PS_SMALL;
            if (large && n != 1) return "a large front is an item alone";
            *n_large += large;
            if (depth[s] != depth[tq_sn[tq_ptr[q]]]) return "one depth per item";
        }
    }
    for (int s = 0; s < fr.S; ++s)
        for (int k = fr.cptr[s]; k < fr.cptr[s + 1]; ++k)
            if (item[fr.child[k]] >= item[s]) return "children before parents";
    return "";
}

// The pull lists of the forward solves' child gather: summing a front's lists in
// order gives bitwise the child-by-child scatter into zeroed storage.  stride 1:
// one entry per node (the supernodal sweep's d4 vectors, aoff in nodes); stride
// 3: three floats per node (the multifrontal solve, aoff in floats, padded).
static const char* check_pull(const HostFronts& fr, const std::vector<int>& aoff, int stride, long long acc_len) {
    std::vector<int> off, ptr, idx;
    dc_build_pull_lists(fr, aoff, stride, off, ptr, idx);
    std::vector<double> acc(acc_len);
    unsigned long long st = 12345;
    for (double& a : acc) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        a = (double)(long long)(st >> 11) * 0x1.0p-40 - 4096.0;
    }
    for (int s = 0; s < fr.S; ++s) {
        const int fs = fr.f[s] / 3;
        for (int comp = 0; comp < stride; ++comp) {
            std::vector<double> scat(fs, 0.0);
            for (int q = fr.cptr[s]; q < fr.cptr[s + 1]; ++q) {
                const int c = fr.child[q];
                for (int k = fr.uptr[c]; k < fr.uptr[c + 1]; ++k)
                    scat[fr.cmap[k]] += acc[aoff[c] + stride * (k - fr.uptr[c]) + comp];
            }
            for (int t = 0; t < fs; ++t) {
                double x = 0.0;
                for (int e = ptr[off[s] + t]; e < ptr[off[s] + t + 1]; ++e) x += acc[idx[e] + comp];
                if (x != scat[t]) return "pull gather differs from the scatter";
            }
        }
    }
    return "";
}

#define REQUIRE(cond, msg)                         \
    do {                                           \
        if (!(cond)) {                             \
            std::printf("FAIL %s\n", msg);         \
            return 1;                              \
        }                                          \
    } while (0)

int main() {
    const int sizes[3] = {5, 9, 7};
    std::vector<HostMesh> H(3);
    std::vector<HostFactor> F(3);
    std::vector<HostFronts> R(3);
    std::vector<HostPSolve> PS(3);
    dc_params p{};
    p.k_stretch = 1e3;
    p.k_bend = 1e-3;
    p.density = 0.1;
    p.h = 1.0 / 120.0;
    p.global_solver = 1;
    for (int i = 0; i < 3; ++i) {
        std::vector<double> pos;
        std::vector<int> tri;
        grid(sizes[i], pos, tri);
        std::vector<int> pins;
        if (i == 1) pins = {0, sizes[i] - 1};
        std::string e = dc_build_mesh(H[i], (int)pos.size() / 3, pos.data(), (int)tri.size() / 3, tri.data(),
                                      (int)pins.size(), pins.empty() ? nullptr : pins.data());
        REQUIRE(e.empty(), "mesh");
        std::vector<double> mass(H[i].m);
        for (int l = 0; l < H[i].m; ++l) mass[l] = p.density * H[i].abar[l];
        std::string err;
        REQUIRE(dc_build_factor(H[i], p, mass, F[i], err) == DC_OK, "factor");
        REQUIRE(dc_build_fronts(H[i], F[i], R[i]).empty(), "fronts");
        dc_build_psolve(F[i], R[i], PS[i]);
    }
    std::vector<InstInfo> I;
    HostMesh M;
    dc_merge_meshes(H, I, M);
    const int MF = M.m_free;
    int m = 0, mf = 0, T = 0;
    for (int i = 0; i < 3; ++i) {
        REQUIRE(I[i].fo == mf && I[i].to == T && I[i].ext_off == m, "instance offsets");
        m += H[i].m;
        mf += H[i].m_free;
        T += H[i].T;
    }
    REQUIRE(M.m == m && M.m_free == mf && M.T == T, "merged sizes");
    // int2ext / ext2int are inverse permutations; instance i keeps its own nodes
    std::set<int> seen;
    for (int g = 0; g < M.m; ++g) {
        REQUIRE(M.ext2int[M.int2ext[g]] == g, "inverse permutation");
        seen.insert(M.int2ext[g]);
    }
    REQUIRE((int)seen.size() == M.m, "permutation");
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < H[i].m; ++l) {
            const int g = I[i].map(l, MF);
            REQUIRE(M.int2ext[g] == I[i].ext_off + H[i].int2ext[l], "node map");
            REQUIRE((l < H[i].m_free) == (g < MF), "free nodes first");
            for (int k = 0; k < 3; ++k) REQUIRE(M.rest[3 * g + k] == H[i].rest[3 * l + k], "rest positions");
        }
    for (int i = 0; i < 3; ++i)
        for (int t = 0; t < H[i].T; ++t)
            for (int a = 0; a < 3; ++a)
                REQUIRE(M.tri[3 * (I[i].to + t) + a] == I[i].map(H[i].tri[3 * t + a], MF), "triangles");
    // bending rows follow the merged node order and stay inside their instance
    REQUIRE((int)M.bptr.size() == M.m + 1, "bending rows");
    // factors: rows shifted by the instance's free offset (empty rows with solver 1)
    HostFactor FM;
    dc_merge_factors(F, I, FM);
    REQUIRE(FM.n == MF && (int)FM.fptr.size() == MF + 1, "merged factor");
    // fronts: every parent lies on a higher level, every front is listed once
    HostFronts FR;
    dc_merge_fronts(R, I, MF, FR);
    int S = 0;
    for (int i = 0; i < 3; ++i) {
        REQUIRE(I[i].so == S, "front offsets");
        S += R[i].S;
    }
    REQUIRE(FR.S == S, "front count");
    std::vector<int> cnt(S, 0);
    for (int l = 0; l + 1 < (int)FR.lvl_ptr.size(); ++l)
        for (int q = FR.lvl_ptr[l]; q < FR.lvl_ptr[l + 1]; ++q) {
            const int s = FR.lvl_sn[q];
            cnt[s]++;
            REQUIRE(FR.level[s] == l, "level list");
            if (FR.parent[s] >= 0) REQUIRE(FR.level[FR.parent[s]] > l, "parent above child");
        }
    for (int s = 0; s < S; ++s) REQUIRE(cnt[s] == 1, "each front once");
    for (int i = 0; i < 3; ++i)
        for (int s = 0; s < R[i].S; ++s) {
            const int g = I[i].so + s;
            REQUIRE(FR.begin[g] == R[i].begin[s] + I[i].fo, "front nodes");
            REQUIRE(FR.parent[g] == (R[i].parent[s] < 0 ? -1 : R[i].parent[s] + I[i].so), "front parents");
        }
    int n_large = 0;
    const char* bad = check_items(FR, &n_large);
    REQUIRE(!*bad, bad);
    {
        // one larger cloth, so that fronts of more than DC_PS_SMALL nodes occur
        std::vector<double> pos;
        std::vector<int> tri;
        grid(40, pos, tri);
        HostMesh h;
        HostFactor hf;
        HostFronts hr;
        REQUIRE(dc_build_mesh(h, (int)pos.size() / 3, pos.data(), (int)tri.size() / 3, tri.data(), 0, nullptr)
                    .empty(),
                "mesh 40");
        std::vector<double> mass(h.m);
        for (int l = 0; l < h.m; ++l) mass[l] = p.density * h.abar[l];
        std::string err;
        REQUIRE(dc_build_factor(h, p, mass, hf, err) == DC_OK, "factor 40");
        REQUIRE(dc_build_fronts(h, hf, hr).empty(), "fronts 40");
        int nl = 0;
        bad = check_items(hr, &nl);
        REQUIRE(!*bad, bad);
        REQUIRE(nl > 0, "large fronts in the 40 x 40 cloth");
    }
    // supernodal panels: offsets concatenated in instance order
    HostPSolve PM;
    dc_merge_psolve(PS, PM);
    REQUIRE((int)PM.poff.size() == S, "panel offsets");
    size_t panel = 0;
    for (int i = 0; i < 3; ++i) panel += PS[i].panel.size();
    REQUIRE(PM.panel.size() == panel, "panel size");
    for (int i = 0; i < 3; ++i)
        for (int s = 0; s < R[i].S; ++s) {
            const int g = I[i].so + s;
            const int ns = R[i].end[s] - R[i].begin[s];
            for (int k = 0; k < ns; ++k)   // diagonal of the panel = diagonal of L
                REQUIRE(PM.panel[PM.poff[g] + (long)k * (ns + R[i].uptr[s + 1] - R[i].uptr[s]) + k] ==
                            PS[i].panel[PS[i].poff[s] + (long)k * (ns + R[i].uptr[s + 1] - R[i].uptr[s]) + k],
                        "panel values");
        }
    bad = check_pull(FR, PM.aoff, 1, PM.acc_nodes);
    REQUIRE(!*bad, bad);
    std::vector<int> acc_base(FR.S);
    for (int q = 0; q < FR.S; ++q) acc_base[q] = (int)FR.acc_off[q];
    bad = check_pull(FR, acc_base, 3, FR.acc_size);
    REQUIRE(!*bad, bad);
    std::printf("ok %d %d %d\n", M.m, MF, S);
    return 0;
}
