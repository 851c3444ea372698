// Device view and launchers of the adjoint step (see dc_adjoint.cu).
#pragma once

#include "dc_internal.h"

struct AdjDev {
    double h;
    const double* mu;     // [m] friction coefficient of each node's instance
    d4* tr0;              // [T] (R col 0, S^-1_00)
    d4* tr1;              // [T] (R col 1, S^-1_01)
    d4* tr2;              // [T] (S^-1_11, 1/tr S, P_12, P_22)
    d4* tav;              // [4T] per triangle: a_v (xyz) of its 3 vertices, then (P_00, P_01, P_02, P_11);
                          // a_v = (g_v0 R1 - g_v1 R0) / tr S, P = I - R0 R0^T - R1 R1^T
    d4* bq;               // [m] (q_hat, s/|q|)
    d4* dinv;             // [3 m_free] rows of the constrained block inverse D+
    d4* slip;             // [m_free] (t_hat, h mu f_N / |u_T|) for slip nodes
    int* type;            // [m_free] 0 free / take-off, 1 stick, 2 slip
    const int* contact;   // step record: obstacle index or -1
    const int* case_;     // step record: 0 take-off, 1 stick, 2 slip
    const d4* nb;         // step record: (normal, beta)
    const d4* f;          // step record: contact force
    const int* node_inst; // [m] instance of each node
    const double* mask;   // [n_inst] or NULL: instances with mask 0 are skipped (their
                          // outputs keep stale, finite values that are only ever scaled by 0)
    d4* c1;               // element-pass scratch [T]
    d4* c2;               // [T]
    d4* bu;               // [m]
};

void adj_setup(const DevMesh& dm, const AdjDev& ad, const d4* x1, const d4* v1, cudaStream_t s);
void adj_rhs(const DevMesh& dm, const AdjDev& ad, const d4* gx, const d4* gv, d4* g, d4* rhs, cudaStream_t s);
// mode 0: out = Pi_B H z; 1: out = w - Pi_B H z; 2: out = w - H z; 3: out = h^2 grad^2 W z on all nodes
void adj_apply_H(const DevMesh& dm, const AdjDev& ad, int mode, const d4* z, const d4* w, d4* out, cudaStream_t s);
void adj_dplus(const DevMesh& dm, const AdjDev& ad, const d4* base, const d4* w, d4* out, cudaStream_t s);
void adj_solve_project(const DevMesh& dm, const AdjDev& ad, const d4* r, d4* ytmp, const d4* base, d4* out,
                       cudaStream_t s);
// Per-instance reduction layout of a context (see the Krylov helpers).
struct Segs {
    int B = 0, nchunk = 0, npchunk = 0;
    const int4* chunk = nullptr;     // [nchunk] (inst, lo, hi, -) in doubles of the free-node vectors
    const int* cptr = nullptr;       // [B + 1] chunks of instance i
    const int4* pchunk = nullptr;    // [npchunk] (inst, kind, lo, hi) element ranges of the parameter terms
    const int* pcptr = nullptr;      // [3 B + 1] chunks of (instance i, kind q) at 3 i + q
};
// out[j * B + i] = V_j . w over instance i's free nodes, j < nvec
// clist (optional): device list of the ncl chunks to process (others keep stale
// partial sums / values that callers must not use).
void adj_bdot(const Segs& sg, const double* V, long ldv, int nvec, const double* w, double* partial, double* out,
              cudaStream_t s, const double* mask = nullptr, const int* clist = nullptr, int ncl = 0);
// w += sign * sum_j V_j coef[j * B + i] on instance i's free nodes
void adj_bvupdate(const Segs& sg, const double* V, long ldv, int nvec, const double* coef, double* w, double sign,
                  cudaStream_t s, const double* mask = nullptr, const int* clist = nullptr, int ncl = 0);
// out = a * sc[i] on instance i's free nodes (exactly 0 where sc[i] == 0)
void adj_bscale(const Segs& sg, const double* a, const double* sc, double* out, cudaStream_t s,
                const int* clist = nullptr, int ncl = 0);
void adj_outputs(const DevMesh& dm, const AdjDev& ad, const DevParams& P, const d4* z, const d4* E,
                 const d4* resid, const d4* x_n, const d4* v1, const d4* gx, d4* gx_out, d4* gv_out,
                 cudaStream_t s);
// acc[4 i + q] += dL/d(k_stretch, k_bend, mu)_q of instance i for this step
void adj_params(const DevMesh& dm, const AdjDev& ad, const Segs& sg, const d4* z, const d4* x1, double* part,
                double* acc, cudaStream_t s);
// g += the caller-order array ext (layout DC_LAYOUT_*), permuted to internal order
void adj_add_ext(d4* g, const double* ext, const int* int2ext, int m, int layout, cudaStream_t s);

// Per-step multifrontal LDL^T preconditioner (dc_frontal.cu).
size_t frontal_factor_smem(int max_f, int max_p, bool tc);
bool frontal_level_tc(int max_f);
dc_status frontal_debug_factor(int n, int p, const float* A, float* out, float* linv_out, int threads, int tc,
                               int use_gscr, std::string* err);
// a factorisation CTA with its panel scratch in global memory: shared bytes, and
// global floats per CTA
size_t frontal_factor_smem_small(bool tc);
long frontal_factor_gscr(int max_f, int max_p);
size_t frontal_solve_smem(int max_f);
// Raises the shared-memory limits of the factorisation kernel (to factor_bytes)
// and of the solve kernels (fronts of up to max_f unknowns).
cudaError_t frontal_configure(size_t factor_bytes, int max_f);
// Fronts per level that exceed the shared memory of one CTA: the global scratch
// (floats) their level launch needs, the largest over the levels (0 if none),
// and the largest shared-memory size of the other levels.
void frontal_plan(const HostFronts& fr, size_t smem_limit, long* gscr_floats, size_t* factor_bytes);
// Launch shape of the tree-scheduled solves for fronts of at most max_f
// unknowns: the CTAs of each kernel that fit on the device at once, and the
// dynamic shared memory.
cudaError_t frontal_tree_grid(int max_f, int* grid_f, int* grid_b, size_t* smem);
// lvl_ptr / lvl_maxf / lvl_maxp: host arrays, the fronts of level l are
// lvl_sn[lvl_ptr[l] .. lvl_ptr[l+1]), the largest has lvl_maxf[l] unknowns and
// the largest pivot block lvl_maxp[l].
void frontal_factorize(const DevMesh& dm, const AdjDev& ad, const FrontDev& fd, const int* lvl_ptr, int nlev,
                       const int* lvl_maxf, const int* lvl_maxp, cudaStream_t s, KTimer* kt = nullptr);
// act_sn / act_ptr (optional): device list of the fronts to solve, level l at
// act_sn[act_ptr[l] .. act_ptr[l+1]) (act_ptr on the host); fronts of masked
// instances may be listed (they exit at once), active ones must be.  With
// fd.tree the two solves are one launch each over act_tq[0 .. n_act_tq) (the
// same fronts in fd.tq's order), or over fd.tq when act_tq is null.
void frontal_precond(const AdjDev& ad, const FrontDev& fd, const int* lvl_ptr, int nlev, const int* lvl_maxf,
                     int n_free, const d4* w, d4* out, cudaStream_t s, KTimer* kt = nullptr,
                     const int* act_sn = nullptr, const int* act_ptr = nullptr, const int* act_tq = nullptr,
                     int n_act_tq = 0);
