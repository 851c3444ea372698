// Internal declarations shared by the host setup, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dc.h"

// A node vector record: (x, y, z, pad).  Node vectors are read by index (by
// triangles, bending stencils and the solve), so one 32-byte record is a single
// sector per gather.
struct __align__(32) d4 {
    double x, y, z, w;
};

// Host-side count of kernel launches made by the library (all contexts).
void dc_note_launch();
void dc_add_launches(long long n);
long long dc_launch_count();

// CUDA-event timing of one kernel class on a context's stream (classes: DC_KT_*).
struct KTimer {
    int cls = 0;
    cudaStream_t stream = nullptr;
    std::vector<cudaEvent_t> ev;
    int used = 0;
    double ms = 0.0;
    long long launches = 0;
    void begin(int c);
    void end(int c);
    void flush();
    void release();
};

// ---------------------------------------------------------------- host setup

struct HostMesh {
    int m = 0, T = 0, m_free = 0;
    // node numbering: internal index = position in (ND order of free nodes, then pins)
    std::vector<int> ext2int, int2ext;
    std::vector<double> rest;          // [m][3], internal order
    // triangles (internal node indices)
    std::vector<int> tri;              // [T][3]
    std::vector<double> G;             // [T][4]: rows 1 and 2 of G = E Dm^-1 (row 0 = -(row1+row2))
    std::vector<double> area;          // [T]
    // bending stencil rows l_b (CSR over vertices, internal indices, self included)
    std::vector<int> bptr, bidx;
    std::vector<double> bval;
    std::vector<double> abar, sb;      // [m]
    std::vector<double> qrest;         // [m][3]
    // ND tree levels per free node (depth of its separator / leaf) and block id
    std::vector<int> nd_level, nd_block;
    int nd_depth = 0;
};

// Builds rest operators and the nested-dissection ordering.  Returns "" or an error.
std::string dc_build_mesh(HostMesh& hm, int n_nodes, const double* rest_pos, int n_tris,
                          const int32_t* tris, int n_pins, const int32_t* pins);

// Sparse lower-triangular factor in CSC (row indices ascending, diagonal first).
struct HostFactor {
    int n = 0;
    std::vector<int> colptr, rowidx;
    std::vector<double> val;
    std::vector<int> parent;           // elimination tree
    // L^-1 as CSR by rows (forward solve) and L^-T as CSR by rows (backward solve)
    std::vector<int> fptr, fidx;
    std::vector<double> fval;
    std::vector<int> bptr, bidx;
    std::vector<double> bval;
    double max_diag = 0.0;             // largest diagonal entry of P_ff
    std::vector<double> pdiag;         // diagonal of P_ff
};

// Diagonal of P_ff^-1 from the factor's CSC columns (rowidx / val still held):
// the selected inverse Z = P^-1 on the pattern of L, computed column by column
// from the last (Takahashi's recurrence for P = L L^T):
//   Z_ij = -(1/L_jj) sum_{k in struct(j)} L_kj Z_ik   (i in struct(j))
//   Z_jj = 1/L_jj^2 - (1/L_jj) sum_{k in struct(j)} L_kj Z_kj.
void dc_inverse_diagonal(const HostFactor& hf, std::vector<double>& zdiag);

// Assembles P_ff (free nodes, internal order) and factorises it.  Returns
// DC_OK, DC_ERR_NOT_SPD or DC_ERR_INVALID with a message in err.  symbolic_only:
// the elimination tree and the structure of L (colptr, rowidx) without values
// (the numeric factorisation then runs on the GPU).
dc_status dc_build_factor(const HostMesh& hm, const dc_params& p, const std::vector<double>& mass,
                          HostFactor& hf, std::string& err, bool symbolic_only = false);

// Symbolic structure of the per-step multifrontal LDL^T (dc_frontal_setup.cpp).
struct HostFronts {
    int S = 0, max_f = 0;
    std::vector<int> begin, end, parent, level, f, p;
    std::vector<long long> off, acc_off, binv_off, linv_off;
    long long pool_size = 0, acc_size = 0, binv_size = 0, linv_size = 0;
    std::vector<int> uptr, unode, cptr, child, cmap, lvl_ptr, lvl_sn;
    std::vector<int> pr_i, pr_j, pr_ld, pr_cptr, pr_code;
    std::vector<long long> pr_dst;
    std::vector<double> pr_coef;
};
std::string dc_build_fronts(const HostMesh& hm, const HostFactor& hf, HostFronts& fr);

// Dense supernodal storage of the scalar factor L of P (global_solver 1), on the
// supernode partition of the fronts: supernode s has ns = (end - begin) nodes and
// nu update rows U_s; its panel is L's columns begin..end-1 restricted to the rows
// (s's nodes, U_s), (ns + nu) x ns column-major, and xinv holds the inverse of
// the panel's ns x ns lower-triangular top block, column-major.  The backward
// sweep reads transposed copies (pant: L_Us^T, ns x nu; xinvt: the inverse
// transposed), so that both sweeps are column-major products.
struct HostPSolve {
    std::vector<long long> poff, xoff;   // [S] offsets of panel / inverse (doubles)
    std::vector<long long> toff;         // [S] offset of the transposed update block (doubles)
    std::vector<int> aoff;               // [S] offset of the update vector (nodes)
    std::vector<double> panel, xinv, pant, xinvt;   // empty when the GPU fills them
    long long n_panel = 0, n_xinv = 0, n_pant = 0;  // their sizes (doubles)
    long long acc_nodes = 0;
};
// values = false: offsets and sizes only (the GPU factorisation fills the panels)
void dc_build_psolve(const HostFactor& hf, const HostFronts& fr, HostPSolve& ps, bool values = true);
void dc_merge_psolve(const std::vector<HostPSolve>& P, HostPSolve& out);
// Work items of the tree-scheduled sweeps (see PSolveDev::tq_ptr)
void dc_build_tree_items(const HostFronts& fr, std::vector<int>& tq_ptr, std::vector<int>& tq_sn);
// Pull lists of the forward solves' child gather (see PSolveDev::pull_off and
// FrontDev::pull_off): entry j of child c's update vector is aoff[c] + stride j
void dc_build_pull_lists(const HostFronts& fr, const std::vector<int>& aoff, int stride, std::vector<int>& pull_off,
                         std::vector<int>& pull_ptr, std::vector<int>& pull_idx);

// ---------------------------------------------------------------- device views

// Supernodal substitution: fronts of at most this many nodes are solved by one
// warp each, larger ones by a whole CTA.
constexpr int DC_PS_SMALL = 64;
// small fronts solved together by one CTA (one per warp)
constexpr int DC_PS_WARPS = 8;

// Device view of the supernodal substitution (global_solver 1): the front
// partition (node-level counts are the fronts' DOF counts / 3) and the panels.
struct PSolveDev {
    int nlev;
    // level l's fronts are sn[lvl_ptr_h[l] ..): first nbig_h[l] large ones (CTA
    // path, the largest maxbig_h[l] nodes), then nsmall_h[l] small ones (warp path)
    const int* lvl_ptr_h;              // host
    const int* nbig_h;                 // host
    const int* nsmall_h;               // host
    const int* maxbig_h;               // host
    const int* sn;
    const int* begin;
    const int* f;                      // DOFs of the front (3 per node)
    const int* p;
    const int* uptr;
    const int* unode;
    const int* cptr;
    const int* child;
    const int* cmap;
    const long long* poff;
    const long long* xoff;
    const long long* toff;
    const int* aoff;
    const double* panel;
    const double* xinv;
    const double* pant;
    const double* xinvt;
    d4* acc;                           // update vectors of the forward sweep (nodes)
    d4* xint;                          // solution of the backward sweep before any per-node update
    // tree-scheduled sweeps (one launch per sweep): work items in a topological
    // order, children first; item q is the fronts tq_sn[tq_ptr[q] .. tq_ptr[q+1]),
    // one large front or up to DC_PS_WARPS small ones of equal depth
    int tree;                          // 1: tree-scheduled sweeps, 0: one launch per level
    int S, n_items;
    const int* parent;                 // [S] parent front, -1 at a root
    const int* tq_ptr;
    const int* tq_sn;
    // gather of the children's update vectors into front s: position t < fs/3
    // sums acc[pull_idx[e]] for e in [pull_ptr[pull_off[s] + t], pull_ptr[pull_off[s] + t + 1]),
    // children in cptr order
    const int* pull_off;               // [S]
    const int* pull_ptr;
    const int* pull_idx;
    int* sched;                        // [2][S + 1]: ticket counter, then per-front done flags (fwd; bwd)
    unsigned long long* fault;         // sticky: set when a dependency wait gave up
    int tree_grid_f, tree_grid_b;      // host: CTAs of a tree-scheduled launch (fwd, bwd)
    size_t tree_smem;                  // host: its dynamic shared memory
    int fused;                         // host: 1: both sweeps of a global step as one launch
};

struct DevMesh {
    int m, m_free, T;
    int solver;                        // 0: explicit inverse rows; 1: supernodal (ps)
    PSolveDev ps;
    const int4* tri;                   // [T] (i0, i1, i2, 0)
    const d4* G;                       // [T] (g1x, g1y, g2x, g2y)
    const double* wt;                  // [T] k_stretch * area
    const double* area;                // [T]
    const int* bptr;                   // bending stencil rows (CSR over m vertices)
    const int* bidx;
    const double* bval;
    const double* wb;                  // [m] k_bend * abar
    const double* abar;                // [m]
    const double* sb;                  // [m]
    const d4* qrest;                   // [m]
    const double* mass;                // [m]
    const int* iptr;                   // node -> triangle incidences (t*3 + a)
    const int* iidx;
    const int* tbptr;                  // node j -> bending rows b containing j, with l_bj
    const int* tbidx;
    const double* tbval;
    const int* fptr;                   // L^-1 rows (CSR), rows 0..m_free-1
    const int* fidx;
    const double* fval;
    int n_long, n_short;               // L^-1 rows split by length (CTA / warp per row)
    const int* long_rows;
    const int* short_rows;
    const int* kptr;                   // L^-T rows (CSR)
    const int* kidx;
    const double* kval;
    // threads per block of the element / node kernels (picked by the autotuner;
    // no launch shape changes any result)
    int bs_local, bs_gather, bs_elem, bs_node;
};

// Parameters seen by the kernels.  h, gravity and the contact margin are shared
// by every instance of a context; friction and obstacles are per instance
// (node -> instance -> table), the stiffnesses are folded into DevMesh::wt/wb.
struct DevParams {
    double h;
    double g[3];
    double delta;
    int compliance;                    // DC_COMPLIANCE_* of the context
    int mass_split;                    // 1: the global step is the mass splitting (DC_COMPLIANCE_MASS)
    const double* ccon;                // [m_free] constant compliance (every mode but ROWSUM)
    const int* node_inst;              // [m] instance of each internal node
    const double* node_mu;             // [m] friction coefficient of the node's instance
    const int* optr;                   // [n_inst + 1] obstacles of instance i: optr[i] .. optr[i+1]-1
    const int* okind;                  // [n_obst] DC_PLANE / DC_SPHERE / DC_CAPSULE / DC_MESH
    const double* oprm;                // [n_obst][8] obstacle parameters (normalised plane; for a
                                       // mesh: first triangle record, triangle count)
    const d4* mesh;                    // triangle records of the context's meshes (dc_obstacle.cuh)
};

// Instance layout inside a context.  Internal node order is: the free nodes of
// instance 0, 1, ... (each in its own nested-dissection order), then the pinned
// nodes of instance 0, 1, ...; external (caller) node order is the concatenation
// of the instances' own numberings.
struct InstInfo {
    int m = 0, mf = 0, T = 0;          // nodes, free nodes, triangles
    long long ext_off = 0;             // first external node
    int fo = 0;                        // first internal free node
    int po = 0;                        // first pinned node, relative to the total free count
    int to = 0;                        // first triangle
    int so = 0;                        // first supernode of the adjoint fronts
    int map(int l, int MF) const { return l < mf ? fo + l : MF + po + (l - mf); }
};

// Concatenates per-instance meshes into one disconnected mesh (fills the offsets).
void dc_merge_meshes(const std::vector<HostMesh>& H, std::vector<InstInfo>& I, HostMesh& out);
// Concatenates per-instance factors (explicit inverse rows only) with node offsets.
void dc_merge_factors(const std::vector<HostFactor>& F, const std::vector<InstInfo>& I, HostFactor& out);
// Concatenates per-instance front structures; levels are merged by height.
void dc_merge_fronts(const std::vector<HostFronts>& F, std::vector<InstInfo>& I, int MF, HostFronts& out);

// ---------------------------------------------------------------- kernel launchers
// (all asynchronous on the given stream)

// layout: DC_LAYOUT_NODE_MAJOR ([m][3]) or DC_LAYOUT_COMPONENT_MAJOR ([3][m]) of ext
void launch_permute_in(const double* ext, d4* out, const int* ext2int, int m, int layout, cudaStream_t s);
void launch_permute_out(const d4* in, double* ext, const int* int2ext, int m, int layout, cudaStream_t s);
void launch_zero_pins(d4* v, int m_free, int m, cudaStream_t s);

// contact detection + per-step constants (Sec. 3.2, reading R4)
void launch_detect(const DevMesh& dm, const DevParams& P, const d4* x_n, const d4* v_n,
                   int* contact, d4* normal_beta, d4* f, d4* ind, cudaStream_t s);
// local step over triangles and bending vertices (Sec. 3.1)
void launch_local(const DevMesh& dm, const DevParams& P, const d4* x_n, const d4* v,
                  d4* tri_c1, d4* tri_c2, d4* bend_u, cudaStream_t s);
// right-hand side gather: b = M (v_n + h g) + sum contributions + h f
void launch_gather_rhs(const DevMesh& dm, const DevParams& P, const d4* v_n, const d4* tri_c1,
                       const d4* tri_c2, const d4* bend_u, const d4* f, d4* b, cudaStream_t s);
// forward solve y = L^-1 b
void launch_solve_fwd(const DevMesh& dm, const d4* b, d4* y, cudaStream_t s);
// backward solve out = L^-T y; mode 0: plain output; mode 1: output then per-node
// Signorini-Coulomb update (writes v, f, case); mode 2: compliance c_j = h * out_j.x
void launch_solve_bwd(const DevMesh& dm, const DevParams& P, const d4* y, d4* out, int mode,
                      const int* contact, const d4* normal_beta, const double* c, d4* f,
                      int* case_, double* c_out, cudaStream_t s);
// Both substitution sweeps of one global step as one tree-scheduled launch (the
// forward sweep, then launch_solve_bwd's backward sweep with the same mode and
// outputs), when global_solver 1 runs tree-scheduled with fused sweeps; returns
// false (nothing launched) otherwise.
bool launch_solve_sweeps(const DevMesh& dm, const DevParams& P, const d4* b, d4* y, d4* out, int mode,
                         const int* contact, const d4* nb, const double* c, d4* f, int* case_, double* c_out,
                         cudaStream_t s);
// Raises the shared-memory limit of the supernodal level kernels for fronts of
// up to max_fs nodes (process-wide, never lowered).
cudaError_t psolve_configure(int max_fs);
// The tree-scheduled forward sweep with its first `skip` tickets taken before
// the launch (testing the bounded waits: those items never run).
void launch_solve_fwd_skip(const DevMesh& dm, const d4* b, d4* y, int skip, cudaStream_t s);
// Launch shape of the tree-scheduled sweeps whose largest CTA-path front has
// max_fs nodes: the CTAs of each kernel that fit on the device at once, and the
// dynamic shared memory
cudaError_t psolve_tree_grid(int max_fs, int* grid_f, int* grid_b, size_t* smem);
// x_{n+1} = x_n + h v; sets *nonfinite when a state entry is not finite
void launch_finalize(const DevMesh& dm, const DevParams& P, const d4* x_n, const d4* v,
                     d4* x_np1, unsigned long long* nonfinite, cudaStream_t s);
// Instances whose step count inst_steps[i] <= step keep their state: x_out = x_in,
// v_out = v_in, and their free nodes leave the contact record (contact = -1).
void launch_freeze(const DevMesh& dm, const DevParams& P, const int* inst_steps, int step, const int* step_base,
                   const d4* xin, const d4* vin, d4* xout, d4* vout, int* contact, cudaStream_t s);
void launch_set_int(int* p, int v, cudaStream_t s);
// gv_out = gv_in on the nodes of instances with inst_steps[i] <= step (their
// adjoint passes through a step they did not take).
void launch_pass_adjoint(const DevMesh& dm, const DevParams& P, const int* inst_steps, int step, const d4* gv_in,
                         d4* gv_out, cudaStream_t s);
// Global step of the mass splitting (DC_COMPLIANCE_MASS): v_half = M^-1 b per
// free node, then the node's Signorini-Coulomb update as in launch_solve_bwd mode 1
void launch_mass_solve(const DevMesh& dm, const DevParams& P, const d4* b, d4* v, const int* contact,
                       const d4* normal_beta, const double* c, d4* f, int* case_, cudaStream_t s);
void launch_count_cases(const int* contact, const int* case_, int m_free,
                        unsigned long long* counters, cudaStream_t s);

// Device view of the multifrontal structure and its per-step numeric storage.
struct FrontDev {
    int S, NP, max_f;
    const float* tau;                  // [S] pivots below tau[s] are replaced by +-tau[s]
    const int* sn_inst;                // [S] instance of each front
    long long pool_size;
    const int* begin;
    const int* f;
    const int* p;
    const long long* off;
    const long long* acc_off;
    const long long* binv_off;         // per front: offset of its diagonal-block inverses
    const long long* linv_off;         // per front: offset of the inverse of its pivot block
    const int* uptr;
    const int* unode;
    const int* cptr;
    const int* child;
    const int* cmap;
    const int* lvl_sn;
    const int* pr_i;
    const int* pr_j;
    const long long* pr_dst;
    const int* pr_ld;
    const int* pr_cptr;
    const int* pr_code;
    const double* pr_coef;
    float* pool;                       // fronts (lower triangles used)
    float* acc;                        // per-front update vectors of the forward solve
    float* binv;                       // inverses of the 32x32 unit-lower diagonal blocks
    float* linv;                       // inverses of the unit-lower pivot blocks (p x p, column-major)
    float* rvec;                       // [3 m_free] right-hand side
    float* zvec;                       // [3 m_free] D^-1 L^-1 r
    float* xvec;                       // [3 m_free] solution
    // tree-scheduled solves (one launch per sweep): the fronts in a topological
    // order (children first), their parents, and the launches' ticket counters
    // and done flags
    int tree;                          // 1: tree-scheduled solves, 0: one launch per level
    // gather of the children's update vectors into front s: node t < f/3 sums the
    // 3-float entries acc[pull_idx[e] ..] for e in [pull_ptr[pull_off[s] + t],
    // pull_ptr[pull_off[s] + t + 1]), children in cptr order
    const int* pull_off;               // [S]
    const int* pull_ptr;
    const int* pull_idx;
    const int* tq;                     // [S]
    const int* parent;                 // [S] -1 at a root
    int* sched;                        // [2][S + 1]: ticket, then per-front done flags (fwd; bwd)
    unsigned long long* fault;         // sticky: set when a dependency wait gave up
    int tree_grid_f, tree_grid_b;      // host: CTAs of a tree-scheduled launch
    size_t tree_smem;                  // host: its dynamic shared memory
    // factorisation levels whose CTAs need more than smem_limit bytes of shared
    // memory keep their panel scratch in gscr instead (per CTA, per slot)
    size_t smem_limit;                 // host
    float* gscr;
};
