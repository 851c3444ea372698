/*
 * dc.h -- C ABI of the GB300 differentiable-cloth library (libdc.so).
 *
 * One Projective Dynamics (PD) cloth time step with dry frictional
 * (Signorini-Coulomb) contact, and its adjoint, after "DiffCloth:
 * Differentiable Cloth Simulation with Dry Frictional Contact"
 * (arXiv 2106.05306), Sec. 3-4.
 *
 * Conventions for every entry point
 *  - Functions return a dc_status (0 = DC_OK) and never throw.  dc_last_error()
 *    gives a message for the last failing call on a context.
 *  - Node arrays are FP64 in the node numbering of the mesh passed to
 *    dc_create_mesh, node-major "[m][3]" (x0,y0,z0,x1,...) by default, or
 *    component-major "[3][m]" (all x, then all y, then all z) after
 *    dc_set_layout(ctx, DC_LAYOUT_COMPONENT_MAJOR).
 *  - Array arguments may be host or device pointers (CUDA unified addressing
 *    tells them apart).  Device pointers keep the call asynchronous on the
 *    context's stream; if any argument is host memory the call synchronises the
 *    stream before it returns.  The caller owns every argument array; the
 *    library owns the factor, work buffers and checkpoints.
 *  - All GPU work is enqueued on the CUDA stream given to dc_create_mesh.
 *    Errors found on the device are reported by the next synchronising call
 *    (dc_sync, dc_get_stats, dc_backward, or any call with host buffers): a
 *    non-finite state at the end of a forward step as DC_ERR_NONFINITE (reported
 *    once); and a triangular-solve sweep over the elimination trees (the
 *    supernodal substitution of global_solver 1, the preconditioner solves of
 *    the adjoint) is one launch whose CTAs wait for one another's fronts, every
 *    such wait is bounded, and one that gives up sets a sticky device flag
 *    reported as DC_ERR_TIMEOUT (the context's results are invalid from then on).
 *  - A context is not thread-safe.
 *  - Batches.  dc_create_batch packs several cloths (instances) of any sizes
 *    into one context; every call below then works on all of them at once,
 *    with one kernel launch per phase covering every instance.  Node arrays
 *    are the concatenation of the instances' [m_i][3] arrays in instance order
 *    (dc_get_layout gives the offsets) and dL_dparams holds 3 values per
 *    instance.  An instance's results do not depend on the other instances of
 *    its batch: they are bitwise those of a one-instance context of that cloth.
 */
#ifndef DC_H_
#define DC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dc_status;
enum {
    DC_OK = 0,
    DC_ERR_INVALID = 1,      /* bad size, index, pointer or parameter (host check) */
    DC_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    DC_ERR_NOT_SPD = 3,      /* the PD matrix factorisation met a pivot <= 0 */
    DC_ERR_OOM = 4,          /* device allocation failed */
    DC_ERR_NONFINITE = 5,    /* a NaN/Inf was produced on the device */
    DC_ERR_NONCONVERGED = 6, /* an adjoint step stopped above adj_tol (after its fallback) */
    DC_ERR_STATE = 7,        /* call out of order (e.g. dc_step before dc_set_params) */
    DC_ERR_TIMEOUT = 8       /* a bounded device-side wait gave up (see above) */
};

/* Compliance c_j of the per-node contact solve (Eq. ly_et_al_govrningEq: the
 * Signorini-Coulomb law is solved per node against a diagonal approximation of
 * the velocity response to its impulse, v = v_free + c_j r_j).
 *   DC_COMPLIANCE_ROWSUM (default): c_j = h (P^-1 1_I)_j, the row sum of the
 *       contact block of h P^-1 (one extra P^-1 solve per step).
 *   DC_COMPLIANCE_DIAG_PINV: c_j = h (P^-1)_jj (selected inversion of the factor,
 *       once per dc_set_params).
 *   DC_COMPLIANCE_DIAG_P: c_j = h / P_jj.
 *   DC_COMPLIANCE_MASS: the splitting as printed, M v^{k+1} = b - (P - M) v^k +
 *       h J^T r^{k+1} with c_j = h / m_j: the global step is a per-node division
 *       by the mass instead of P^-1.  It converges only while h^2 rho(M^-1 (P-M)) < 1,
 *       i.e. at small stiffness.
 * Every choice has the same fixed point (Eq. implicit_with_contact); they differ
 * in how fast (and whether) the K PD iterations of a step approach it. */
enum { DC_COMPLIANCE_ROWSUM = 0, DC_COMPLIANCE_DIAG_PINV = 1, DC_COMPLIANCE_DIAG_P = 2, DC_COMPLIANCE_MASS = 3 };

/* Layout of node arrays at the boundary (dc_set_layout). */
enum { DC_LAYOUT_NODE_MAJOR = 0, DC_LAYOUT_COMPONENT_MAJOR = 1 };

enum { DC_PLANE = 0, DC_SPHERE = 1, DC_CAPSULE = 2, DC_MESH = 3 };
#define DC_MAX_OBSTACLES 16

/* Static obstacle (reading of Sec. 3.2 "Extensions": any obstacle with a signed
 * distance; analytic or triangulated, Sec. "Continuity and Smoothness").
 *   DC_PLANE:   p[0..2] = unit normal n, p[3] = d        (surface n.x = d)
 *   DC_SPHERE:  p[0..2] = centre, p[3] = radius
 *   DC_CAPSULE: p[0..2] = a, p[3..5] = b, p[6] = radius  (segment a-b)
 *   DC_MESH:    p[0] = a mesh id from dc_add_obstacle_mesh on the same context */
typedef struct dc_obstacle {
    int32_t kind;
    int32_t pad_;
    double p[7];
} dc_obstacle;

typedef struct dc_params {
    double k_stretch;        /* stretch stiffness; w_t = k_stretch * rest area     */
    double k_bend;           /* bending stiffness; w_b = k_bend * vertex area      */
    double density;          /* kg/m^2; lumped mass = density * vertex area        */
    double mu;               /* Coulomb friction coefficient                       */
    double h;                /* time step (s)                                       */
    double gravity[3];       /* f_ext = M g                                         */
    double contact_margin;   /* detection margin delta (m)                          */
    double adj_tol;          /* adjoint: relative residual target (default 1e-10)   */
    int32_t n_pd_iters;      /* local/global/contact iterations per step (K)       */
    int32_t adj_max_iters;   /* adjoint: cap on preconditioned GMRES iterations     */
    int32_t adj_restart;     /* adjoint: GMRES restart length (<= 256)              */
    int32_t checkpoint_every;/* rollout: keep (x, v) every k steps (>= 1)           */
    int32_t n_obstacles;
    int32_t adj_precond;     /* adjoint preconditioner: 0 = per-step single-precision
                                multifrontal LDL^T of the constrained matrix (default);
                                1 = node-block inverse + projected P^-1 (no factorisation) */
    int32_t global_solver;   /* how P^-1 is applied (Eq. pd_global): 0 = rows of the
                                explicit inverse factors L^-1, L^-T, two launches per
                                application (default; best for one small cloth);
                                1 = supernodal substitution with L, about 4x fewer
                                flops, one launch per sweep with the fronts of the
                                elimination trees taken in dependency order (best for
                                batches; needs adj_precond 0).  Equal results up to
                                rounding. */
    int32_t contact_compliance; /* DC_COMPLIANCE_* (default ROWSUM)                  */
    int32_t adj_fallback;    /* 1 (default): an adjoint step whose GMRES reaches
                                adj_max_iters, or stops more than 100 x adj_tol above
                                it, is solved again by the fallback (dc_backward);
                                0: no fallback                                       */
    int32_t factor_on_gpu;   /* 1: P's numeric Cholesky (Eq. pd_global, "prefactorised")
                                runs on the GPU as a multifrontal FP64 factorisation
                                written straight into the supernodal panels; the host
                                does only the ordering and symbolic analysis.  Needs
                                global_solver 1; not with DC_COMPLIANCE_DIAG_PINV.
                                0 (default): numeric factorisation on the host.      */
    dc_obstacle obstacles[DC_MAX_OBSTACLES];
} dc_params;

typedef struct dc_stats {
    int64_t steps;             /* forward steps run since creation                    */
    int64_t contacts_takeoff;  /* contact-node counts by final case, summed over steps */
    int64_t contacts_stick;
    int64_t contacts_slip;
    int64_t adj_steps;         /* adjoint steps run                                   */
    int64_t adj_iters;         /* preconditioned GMRES iterations, summed             */
    int64_t adj_max_iters_seen;/* largest count in one adjoint step                   */
    int64_t adj_nonconverged;  /* adjoint steps that hit the cap                      */
    double adj_last_residual;  /* relative residual of the last adjoint step          */
    int64_t factor_nnz;        /* nonzeros of the Cholesky factor L of P              */
    int64_t solve_nnz;         /* nonzeros read by one P^-1 application (one column)  */
    int32_t n_free;            /* free (unpinned) nodes                               */
    int32_t nd_levels;         /* depth of the nested-dissection tree                 */
    int64_t kernel_launches;   /* kernels launched by the library (process-wide)      */
    double timer_ms;           /* dc_set_kernel_timer: accumulated device time (ms)   */
    int64_t timer_launches;    /* dc_set_kernel_timer: launches timed                 */
    int64_t fwd_solve_nnz;     /* nonzeros of L^-1 read by one forward substitution   */
    int64_t bwd_solve_nnz;     /* nonzeros of L^-T read by one backward substitution  */
    double front_flops;        /* FP32 flops of one multifrontal factorisation        */
    int32_t front_levels;      /* levels (launches) of one multifrontal factorisation */
    int32_t n_supernodes;      /* supernodes (fronts)                                 */
    int64_t factorisations;    /* multifrontal factorisations run                     */
    int32_t n_instances;       /* cloths packed in the context                        */
    int32_t graphs;            /* 1 if rollouts replay captured CUDA graphs           */
    int64_t graph_replays;     /* CUDA graph launches made                            */
    int32_t block_local;       /* threads per block chosen for the local-step kernel  */
    int32_t block_gather;      /* ... for the right-hand-side and adjoint gathers     */
    int32_t block_node;        /* ... for the per-node kernels                        */
    int32_t block_elem;        /* ... for the adjoint per-element kernel              */
    int64_t adj_batch_iters;   /* GMRES iterations run by a context, all instances in lockstep */
    int32_t global_solver;     /* dc_params.global_solver in use                      */
    int32_t reserved_;
    double psolve_flops;       /* FP64 flops of one supernodal substitution sweep (3 columns) */
    int64_t adj_fallbacks;     /* adjoint steps of one instance re-solved by the fallback */
    int64_t adj_fallback_iters;/* GMRES iterations the fallback solves took            */
    int32_t layout;            /* DC_LAYOUT_* of the node arrays                       */
    int32_t contact_compliance;/* DC_COMPLIANCE_* in use                               */
    int64_t device_bytes;      /* device memory the context holds now                 */
    int64_t device_bytes_peak; /* ... at most since its creation                      */
    int32_t n_nodes;           /* nodes of all instances                              */
    int32_t n_tris;            /* triangles of all instances                          */
    int64_t bend_nnz;          /* entries of the bending stencil rows (all vertices)  */
    int64_t front_entries;     /* FP32 entries stored for one multifrontal factorisation */
} dc_stats;

/* Kernel classes for dc_set_kernel_timer. */
enum {
    DC_KT_NONE = 0,
    DC_KT_SOLVE_FWD = 1,   /* forward substitution of the PD global step (L^-1 rows)   */
    DC_KT_SOLVE_BWD = 2,   /* backward substitution + per-node contact solve           */
    DC_KT_LOCAL = 3,       /* local step (projections)                                 */
    DC_KT_GATHER = 4,      /* right-hand-side gather                                   */
    DC_KT_FRONT = 5,       /* one level of the adjoint multifrontal factorisation      */
    DC_KT_MSOLVE = 6,      /* one level of the multifrontal forward or backward solve  */
    DC_KT_KRYLOV = 7,      /* GMRES vector kernels (dot products, updates, scaling)    */
    DC_KT_APPLYH = 8,      /* adjoint operator application (element pass + gather)    */
    DC_KT_ASSEMBLE = 9,    /* per-step adjoint setup and front assembly               */
    DC_KT_SWEEPS = 10      /* both substitution sweeps of one global step in one launch
                              (global_solver 1; the contact solve fused in)           */
};

typedef struct dc_ctx dc_ctx;

/* Create a cloth from its rest mesh.
 *   rest_pos: [n_nodes][3] rest positions (host).  tris: [n_tris][3] node
 *   indices (host).  pins: [n_pins] node indices held fixed (Dirichlet, velocity
 *   0), may be NULL when n_pins = 0.  stream: a cudaStream_t (NULL = legacy
 *   default stream).  Computes the rest-shape operators of the PD energies
 *   (Sec. 3.1, Eq. pd_project: triangle stretch and vertex bending), the lumped
 *   mass, and a nested-dissection ordering of the free nodes.  The new context
 *   is returned in *out; it must be released with dc_destroy. */
dc_status dc_create_mesh(dc_ctx** out, int32_t n_nodes, const double* rest_pos,
                         int32_t n_tris, const int32_t* tris,
                         int32_t n_pins, const int32_t* pins, void* stream);

/* One cloth of a batch (host arrays, as for dc_create_mesh). */
typedef struct dc_instance {
    int32_t n_nodes;
    int32_t n_tris;
    int32_t n_pins;
    int32_t pad_;
    const double* rest_pos;   /* [n_nodes][3] */
    const int32_t* tris;      /* [n_tris][3]  */
    const int32_t* pins;      /* [n_pins], may be NULL when n_pins = 0 */
} dc_instance;

/* Create one context holding n_instances cloths (n_instances >= 1; DC_ERR_INVALID
 * for an invalid mesh, naming the instance).  The per-instance rest operators
 * and orderings are built on several host threads.  Node numbering: instance i
 * occupies nodes [off_i, off_i + n_nodes_i) of every node array, off_0 = 0. */
dc_status dc_create_batch(dc_ctx** out, int32_t n_instances, const dc_instance* instances,
                          void* stream);

/* Number of instances and, if node_offsets is not NULL, the n_instances + 1
 * node offsets of the concatenated node arrays (host array). */
dc_status dc_get_layout(dc_ctx* ctx, int32_t* n_instances, int64_t* node_offsets);

/* Set material, contact and solver parameters (host struct, copied).
 * Assembles the constant PD matrix P = M + h^2 sum_i w_i A_i^T A_i (Sec. 3.1,
 * Eq. pd_global), factorises it once (P = L L^T, host, nested-dissection
 * order) and uploads the solve operators.  Synchronous.  DC_ERR_NOT_SPD if a
 * pivot is not positive; DC_ERR_INVALID for non-finite or out-of-range values. */
dc_status dc_set_params(dc_ctx* ctx, const dc_params* params);

/* Per-instance parameters of a batch: params[i] for instance i (n_instances
 * entries).  k_stretch, k_bend, density, mu and the obstacles may differ between
 * instances; every other field must be equal in all entries (DC_ERR_INVALID
 * otherwise).  dc_set_params on a batch gives every instance the same values.
 * Each instance's P is assembled and factorised on its own (host threads). */
dc_status dc_set_params_batch(dc_ctx* ctx, int32_t n_instances, const dc_params* params);

/* Per-instance step counts of a batch for the next dc_rollout calls: instance i
 * takes steps[i] steps (0 <= steps[i] <= the n_steps of dc_rollout) and then
 * keeps its state; dc_backward starts its adjoint at the instance's own last
 * step (its adjoint passes unchanged through the steps it did not take).  An
 * instance's results are bitwise those of a rollout of steps[i] steps alone.
 * steps = NULL restores one count for all.  Lets a server pack requests of
 * different lengths into one batch.  No counterpart in the paper. */
dc_status dc_set_instance_steps(dc_ctx* ctx, const int32_t* steps);

/* Register a closed triangle mesh as an obstacle shape of ctx and return its id
 * in *mesh_id, for DC_MESH obstacles of later dc_set_params calls.  verts:
 * [n_verts][3] (host); tris: [n_tris][3] vertex indices (host), counter-clockwise
 * seen from outside; every edge must be shared by exactly two triangles with
 * opposite directions (closed and consistently oriented) and no triangle may be
 * degenerate (DC_ERR_INVALID otherwise).  Its signed distance is |x - c| to the
 * closest surface point c, signed by the angle-weighted pseudo-normal of c's
 * face, edge or vertex, and is computed on the GPU by a closest-triangle query
 * over all its triangles (meant for obstacles of up to a few thousand
 * triangles).  Its normal jumps across edges: the paper's discontinuity of
 * triangulated obstacles (Sec. "Continuity and Smoothness"). */
dc_status dc_add_obstacle_mesh(dc_ctx* ctx, int32_t n_verts, const double* verts, int32_t n_tris,
                               const int32_t* tris, int32_t* mesh_id);

/* Node-array layout of every later call on ctx: DC_LAYOUT_NODE_MAJOR ([m][3],
 * the default) or DC_LAYOUT_COMPONENT_MAJOR ([3][m]: the x block, then y, then
 * z; for a batch m is the total node count and each block is the concatenation
 * of the instances' nodes).  It applies to the state and gradient arguments of
 * dc_step, dc_rollout (traj_x: [(n_steps+1)][3][m]), dc_backward (dL_dtraj_x:
 * [(n_steps+1)][3][m]), dc_global_solve and dc_global_solve_static; dc_create_mesh
 * and dc_create_batch always take [n][3] rest positions.  The conversion is part
 * of the kernels that move node arrays across the boundary (no extra copy).  No
 * counterpart in the paper.  DC_ERR_INVALID for an unknown layout. */
dc_status dc_set_layout(dc_ctx* ctx, int32_t layout);

/* Device bytes a context of these cloths would hold at most through dc_rollout
 * of n_steps steps and dc_backward, computed on the host without touching the
 * device (the meshes are ordered and P factorised on host threads, as
 * dc_create_batch and dc_set_params_batch would): for admission of work by HBM
 * budget.  instances: n_instances cloths (as for dc_create_batch); params: one
 * dc_params per instance.  *bytes receives the total.  DC_ERR_INVALID /
 * DC_ERR_NOT_SPD as dc_create_batch / dc_set_params_batch would report.  No
 * counterpart in the paper. */
dc_status dc_batch_hbm_bytes(int32_t n_instances, const dc_instance* instances, const dc_params* params,
                             int32_t n_steps, int64_t* bytes);

/* Replay the forward steps of dc_rollout and of dc_backward's checkpoint
 * recomputation as captured CUDA graphs (enable = 1) or launch them one by one
 * (0, the default).  A graph is captured on first use for a given step count and
 * replayed afterwards; the results are identical either way.  Graphs are not
 * used while a kernel timer is set, for a trajectory output, or on the legacy
 * default stream (which cannot be captured).  No counterpart in the paper. */
dc_status dc_set_graphs(dc_ctx* ctx, int32_t enable);

/* Time the element and node kernels of the forward step at several block sizes
 * on this context's mesh and keep the fastest (synchronous; reported in
 * dc_stats).  No block size changes any result.  No counterpart in the paper. */
dc_status dc_autotune(dc_ctx* ctx);

/* One time step (x_n, v_n) -> (x_{n+1}, v_{n+1}) (Sec. 3.2, Eq.
 * implicit_with_contact solved by n_pd_iters PD local/global iterations with
 * the per-node Signorini-Coulomb update, Eq. pd_velocity_with_contact).
 * All four arrays are [m][3]; pinned nodes keep their position and get v = 0. */
dc_status dc_step(dc_ctx* ctx, const double* x_n, const double* v_n,
                  double* x_np1, double* v_np1);

/* n_steps time steps from (x0, v0).  Keeps a checkpoint of (x, v) every
 * checkpoint_every steps for dc_backward.  traj_x, if not NULL, receives all
 * positions [(n_steps+1)][m][3] (traj_x[0] = x0). */
dc_status dc_rollout(dc_ctx* ctx, int32_t n_steps, const double* x0, const double* v0,
                     double* x_final, double* v_final, double* traj_x);

/* Gradient of a loss L(x_N, v_N, x_0..x_N) through the last dc_rollout (Sec. 4,
 * Eq. adjoint_v and ppr_adjoint, contact terms as the linearisation of the
 * converged step).  Recomputes each checkpoint segment, then solves one adjoint
 * system per step in reverse order.
 *   dL_dx_final: [m][3] dL/dx_N.  dL_dv_final: [m][3] or NULL (zero).
 *   dL_dtraj_x: [(n_steps+1)][m][3] per-step dL/dx_n or NULL.
 * Outputs dL_dx0, dL_dv0: [m][3]; dL_dparams: [n_instances][3] =
 * dL/d(k_stretch, k_bend, mu) of each instance.
 * Each step's adjoint system is solved by flexible GMRES with the per-step
 * preconditioner (adj_precond); an instance stops at a relative residual of
 * adj_tol, at adj_max_iters, or when a restart cycle no longer halves its
 * residual (the rounding floor of the FP64 operator, about eps cond(H)).  With
 * adj_fallback = 1, an instance that reached adj_max_iters or stopped more than
 * 100 x adj_tol above the tolerance is solved again from its iterate, by
 * GMRES(30) with a stronger preconditioner (the per-step one followed by a
 * sweep of the constrained node-block inverse of H) and a looser stagnation
 * test; the count is in dc_stats.adj_fallbacks.  DC_ERR_NONCONVERGED is
 * reported (after all outputs are written) when an adjoint step still ends
 * above adj_tol. */
dc_status dc_backward(dc_ctx* ctx, const double* dL_dx_final, const double* dL_dv_final,
                      const double* dL_dtraj_x, double* dL_dx0, double* dL_dv0,
                      double* dL_dparams);

/* Per instance of a batch (host array of n_instances entries): the adjoint steps
 * since creation that stopped above adj_tol (the count dc_stats.adj_nonconverged
 * sums), so that a caller can tell which instances a DC_ERR_NONCONVERGED from
 * dc_backward concerns.  The counts are host bookkeeping that dc_backward
 * updates; the call does no device work.  DC_ERR_INVALID on a null argument. */
dc_status dc_get_instance_nonconverged(dc_ctx* ctx, int64_t* counts);

/* Apply P_ff^-1 (the prefactorised global-step matrix restricted to free
 * nodes, Eq. pd_global) to three right-hand-side columns: out = P^-1 rhs.
 * rhs, out: [m][3]; entries of pinned nodes are ignored on input and set to 0. */
dc_status dc_global_solve(dc_ctx* ctx, const double* rhs, double* out);

/* Time every launch of one kernel class (DC_KT_*) with CUDA events recorded on
 * the context's stream; DC_KT_NONE switches timing off.  Resets the
 * accumulated time and count, which dc_get_stats reports.  No counterpart in
 * the paper: measurement support for the roofline report. */
dc_status dc_set_kernel_timer(dc_ctx* ctx, int32_t kernel_class);

/* The same solve as dc_global_solve, for callers that may not allocate device
 * memory while they run: a serving loop that has given the rest of HBM to a
 * caching allocator under a fixed budget, or a latency-bound loop that cannot
 * take the device-wide synchronisation cudaMalloc/cudaFree may cause.  No
 * counterpart in the paper.  It allocates nothing: rhs and out must be device
 * arrays (host pointers are rejected with DC_ERR_INVALID), and its three
 * intermediate node vectors live in a fixed library array of 6 MiB per GPU,
 * held from library load until process exit, which serves meshes of at most
 * 65536 nodes (larger meshes: DC_ERR_INVALID).  The device that was current at
 * dc_create_mesh must be current (DC_ERR_INVALID otherwise); the first call on
 * a device looks up that array's address (cudaGetSymbolAddress); make it before
 * any stream capture.  Every call shares the array: calls that overlap on the
 * GPU (other streams or contexts on the same device) race and must be
 * serialised by the caller.  With global_solver 1 the substitution also writes
 * the context's own sweep vectors and dependency flags (allocated by
 * dc_set_params), so calls on one context must also be serialised with its
 * other calls (the context's stream does that).  Asynchronous on the context's
 * stream. */
dc_status dc_global_solve_static(dc_ctx* ctx, const double* rhs, double* out);

/* Testing the bounded waits of the tree-scheduled sweeps (global_solver 1).
 * Runs one forward supernodal sweep of P^-1 on the context's work vectors with
 * the first skip_items work items never executed, so that a front whose child
 * is among them waits for a flag that nothing sets.  The wait gives up after
 * about a second, sets the context's sticky fault flag and the launch ends; the
 * call synchronises and returns DC_ERR_TIMEOUT when the fault was raised (DC_OK
 * if no skipped item had a waiting parent).  The context's results are invalid
 * afterwards: destroy it.  DC_ERR_INVALID without global_solver 1 or with
 * skip_items outside [1, number of items). */
dc_status dc_debug_sweep_wait_timeout(dc_ctx* ctx, int32_t skip_items);

/* Testing the adjoint preconditioner's dense front kernel on its own: one
 * symmetric n x n front A (host, column-major FP32; the lower triangle is read)
 * with p pivot columns goes through the partial LDL^T that factorises every
 * front of the multifrontal preconditioner (Sec. 4, Eq. ppr_adjoint is the
 * system it preconditions).  out (host, n x n column-major) receives the front
 * afterwards: in its first p columns D on the diagonal and the unit-lower L
 * below it, in the trailing (n - p) x (n - p) lower triangle the Schur
 * complement A22 - L21 D L21^T.  linv_out (host, p x p column-major, nullable)
 * receives the inverse of L's unit-lower pivot block.  threads: 128, 256 or
 * 512; use_tc: 1 updates trailing blocks of 64 rows or more on the tensor
 * cores (TF32 split in three passes, FP32 accumulation), 0 by FP32 FMA tiles;
 * use_gscr: 1 keeps the panel scratch in global memory (the path of fronts
 * too large for shared memory).  Synchronous; allocates its own device memory.
 * DC_ERR_INVALID unless 1 <= p <= n <= 4096 (and the shared memory fits),
 * DC_ERR_TIMEOUT if a tensor-core completion wait gave up, DC_ERR_CUDA on a
 * CUDA error; dc_last_error(NULL) has the message. */
dc_status dc_debug_front_factor(int32_t n, int32_t p, const float* A, float* out, float* linv_out,
                                int32_t threads, int32_t use_tc, int32_t use_gscr);

/* Measured fused-multiply-add throughput of the GPU's CUDA cores, in TFLOP/s
 * (2 flops per FMA), for precision 64 (FP64) or 32 (FP32): a kernel of
 * independent FMA chains on every SM, n_iter x 128 FMAs per chain and thread,
 * best of three launches timed with CUDA events on the current device (legacy
 * default stream, synchronous).  It changes no clock or power setting.  The
 * denominator of the roofline fraction of the ALU-bound kernels.  No
 * counterpart in the paper.  DC_ERR_INVALID for another precision or n_iter < 1. */
dc_status dc_fma_peak(int32_t precision, int32_t n_iter, double* tflops);

/* Counters and factor sizes (synchronises the stream). */
dc_status dc_get_stats(dc_ctx* ctx, dc_stats* out);

/* Wait for all work of the context; reports deferred device errors. */
dc_status dc_sync(dc_ctx* ctx);

/* Release the context and all its device memory (synchronises first). */
void dc_destroy(dc_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing
 * dc_create_mesh when ctx is NULL).  Valid until the next call. */
const char* dc_last_error(dc_ctx* ctx);

/* ------------------------------------------------------------------ serving
 * A request server: many independent forward + adjoint rollouts (each its own
 * cloth, size, step count and parameters) submitted at any time and run
 * concurrently on one GPU.  No counterpart in the paper.
 *  - Each request (or batch of requests, below) is prepared on a host thread
 *    (ordering, factorisation, fronts) as soon as it is submitted, which also
 *    gives its exact device footprint.  It is admitted, in submission order,
 *    when one of n_slots slots is free and its footprint fits in what the HBM
 *    budget has left.  A request larger than the whole budget fails with
 *    DC_ERR_OOM.
 *  - An admitted request keeps its factorisation, fronts and checkpoints
 *    resident until it finishes; slots run on their own CUDA streams and host
 *    threads, so requests overlap on the device, and device memory comes from
 *    the stream-ordered pool (no device-wide synchronisation when a request
 *    starts or ends).
 *  - Continuous batching: with max_batch > 1 a preparation thread packs the
 *    requests queued at that moment whose shared parameters agree (the fields a
 *    batch shares, dc_set_params_batch) into one batch context of up to
 *    max_batch cloths, each with its own step count (dc_set_instance_steps);
 *    a slot runs the whole batch, one launch per phase for all its requests.
 *  - A request's results are bitwise those of the same rollout and backward
 *    run alone through dc_create_mesh / dc_rollout / dc_backward. */
typedef struct dc_server dc_server;

typedef struct dc_server_config {
    int32_t n_slots;           /* requests on the device at once (>= 1)              */
    int32_t n_prep_threads;    /* host threads preparing requests (>= 1)             */
    int64_t hbm_budget_bytes;  /* device bytes the admitted requests may hold        */
    int32_t max_prepared;      /* prepared jobs waiting for a slot, at most          */
    int32_t device;            /* CUDA device ordinal                                */
    int32_t max_batch;         /* requests packed into one batch context (<= 1: one) */
    int32_t reserved_;
} dc_server_config;

typedef struct dc_request {
    int32_t n_nodes, n_tris, n_pins, n_steps;
    const double* rest_pos;      /* [n_nodes][3] host, copied at submission             */
    const int32_t* tris;         /* [n_tris][3]                                         */
    const int32_t* pins;         /* [n_pins] or NULL                                    */
    const double* x0;            /* [n_nodes][3] initial positions                      */
    const double* v0;            /* [n_nodes][3] initial velocities                     */
    const double* dL_dx_final;   /* [n_nodes][3] loss gradient at the last step          */
    const double* dL_dv_final;   /* [n_nodes][3] or NULL                                */
    dc_params params;
} dc_request;

typedef struct dc_result {
    dc_status status;
    int32_t slot;                /* slot that ran the request (-1 if never admitted)    */
    double* x_final;             /* caller-owned [n_nodes][3] host arrays, or NULL:     */
    double* v_final;             /*   filled by dc_server_wait                          */
    double* dL_dx0;
    double* dL_dv0;
    double dL_dparams[3];        /* dL/d(k_stretch, k_bend, mu)                          */
    double t_submit, t_admit, t_done;   /* seconds on the server's clock                */
    int64_t device_bytes;        /* footprint reserved at admission                     */
    int64_t device_bytes_peak;   /* most device memory the request actually held        */
    int64_t adj_iters;           /* GMRES iterations of its adjoint                     */
    char message[256];           /* error message when status != DC_OK                  */
} dc_result;

typedef struct dc_server_stats {
    int64_t submitted, completed, failed;
    int64_t in_flight, peak_in_flight;
    int64_t bytes_reserved, peak_bytes_reserved;
    int64_t cloth_steps;         /* forward steps of the completed requests             */
    int64_t batch_retries;       /* batches that failed and whose requests were run
                                    again one per context (a request that fails alone
                                    no longer takes its batch-mates with it)         */
} dc_server_stats;

/* Start a server (threads and streams) on cfg->device. */
dc_status dc_server_create(dc_server** out, const dc_server_config* cfg);
/* Queue a request (its arrays are copied before the call returns). */
dc_status dc_server_submit(dc_server* srv, const dc_request* req, int64_t* ticket);
/* Wait for a request to finish and collect its results (once per ticket). */
dc_status dc_server_wait(dc_server* srv, int64_t ticket, dc_result* out);
dc_status dc_server_get_stats(dc_server* srv, dc_server_stats* out);
/* Finish every queued request, then stop the threads and free the server. */
void dc_server_destroy(dc_server* srv);

/* Fill *p with the library defaults (k_stretch 1e3, k_bend 1e-3, density 0.1,
 * mu 0.3, h 1/120, g = (0,-9.8,0), delta 1e-6, K = 20, adjoint tol 1e-10,
 * 2000 iterations, restart 200, checkpoint every step, no obstacles,
 * multifrontal preconditioner, ROWSUM compliance, adjoint fallback on). */
void dc_default_params(dc_params* p);

#ifdef __cplusplus
}
#endif
#endif /* DC_H_ */
