"""Plain FP64 CPU oracle: Projective Dynamics cloth time step with dry frictional
(Signorini-Coulomb) contact, and its adjoint (DiffCloth, arXiv 2106.05306).

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference arm import this package.  The CUDA library and its
Python binding never import it, and it imports nothing from them: it shares only
the seeded input generators in ``scenes``.

It is deliberately slow and literal: numpy/scipy, float64, natural node order,
a banded Cholesky of the PD matrix (a different algorithm from the CUDA path's
nested-dissection factor), and a direct sparse LU of the full adjoint KKT
system (the paper treats the direct solve as the ground-truth gradient, Sec. 5.3).

Paper passages followed (section / equation labels of the paper):
  * Sec. 3.1, Eq. implicit_x / implicit_v / implicit_energy: implicit Euler and
    its energy form with y = x_n + h v_n + h^2 M^-1 f_ext.
  * Sec. 3.1, Eq. pd_project / pd_energy / pd_global: PD energies
    W_i = w_i/2 |A_i x - p_i|^2, local projections, and the global system
    P x = M y + h^2 sum w_i A_i^T p_i with constant P = M + h^2 sum w_i A_i^T A_i.
  * Sec. 3.2, Eq. contact_all / implicit_with_contact / pd_velocity /
    pd_velocity_with_contact / ly_et_al_govrningEq: Signorini-Coulomb law and
    the velocity-form global step with the contact impulse h J^T r.
  * Sec. 4.1-4.2, Eq. adjoint / adjoint_pd / adjoint_vv / adjoint_v /
    ppr_adjoint, and "Extensions" (curved obstacles): the adjoint.

Readings of passages the paper leaves open (the CUDA path implements the same ones):
  R1 stretch: A_t maps a triangle to its deformation gradient F = X G (3x2),
     w_t = k_stretch * rest area, projection onto matrices with orthonormal
     columns (the polar factor of F).  A collapsed triangle
     (det F^T F <= 1e-30 (tr F^T F)^2) gets a polar factor built from the
     singular vectors of F with a fixed choice of the missing one, and its
     projection is treated as locally constant in the adjoint (dR = 0).
  R2 bending: A_b is the cotangent Laplacian row of vertex b divided by its
     barycentric area, w_b = k_bend * area, projection onto the sphere of radius
     s_b = |A_b x_rest| (p_b = 0 where the rest shape is flat, s_b = 0).
  R3 lumped mass rho * (1/3 of incident rest area), f_ext = M g, pins are
     Dirichlet (velocity 0, removed from the global system).
  R4 contact set: free nodes whose predicted position x_n + h v_n lies within
     delta of an obstacle (closest obstacle wins, lowest index on ties); normal
     and signed distance are taken at x_n; the Signorini-Coulomb law is imposed
     on the biased normal velocity u_N = n.v + phi(x_n)/h.
  R5 contact iteration: every PD iteration runs local step, global step with
     the previous contact impulse, then an exact per-node closed-form
     Signorini-Coulomb solve with compliance c_j = h * (P^-1 1_I)_j (the row sum
     of the contact block of h P^-1, a Gershgorin bound on the coupling).  The
     printed M-splitting (Eq. ly_et_al_govrningEq) diverges for the stiffness
     values used here; any positive compliance has the same fixed point.
     Alternatives for ablation (params.contact_compliance): "diag_pinv"
     c_j = h (P^-1)_jj, "diag_p" c_j = h / P_jj, and "mass": the splitting as
     printed, M v^{k+1} = b - (P - M) v^k + h J^T r^{k+1} with c_j = h / m_j.
  R7 contact adjoint: the exact linearisation of the converged step, solved as
     one KKT system; stick nodes constrain z_j = 0, slip nodes constrain
     (n - mu t).z_j = 0 (oblique), and the slip friction direction adds
     h mu f_N b b^T / |u_T| to the matrix (the paper's -Delta R).
  R13 node-node self-collision (the J_n paragraph after Eq.
     implicit_with_contact; off unless params.self_thickness > 0): a pair of
     nodes (i, j), i < j, at least one free, sharing no triangle, is in contact
     when their predicted positions are within self_thickness + delta.  Its
     row of J_n acts on the relative velocity v_i - v_j with the normal
     n = (x_i - x_j)/|x_i - x_j| at x_n and the bias beta = (|x_i - x_j| -
     self_thickness)/h, so that an active pair ends at least self_thickness
     apart; the impulse acts as +r on i and -r on j.  As R5's row sum, its
     compliance is the Gershgorin bound of the pairs' coupling,
     c_k = sum_l |h (e_i - e_j)^T P^-1 (e_p - e_q)| over the step's pairs
     l = (p, q) (pinned nodes contribute nothing), which keeps the Jacobi
     iteration over pairs that share nodes from overshooting; when obstacle
     contacts are present as well, each side's bound also counts its coupling
     with the other kind.  Within an
     iteration the pairs are solved from the global step's v_half, Jacobi-style
     beside the obstacle contacts; node i moves by w_i (r_new - r_old) and node
     j by -w_j (r_new - r_old), w_i and w_j proportional to h (P^-1_ii - P^-1_ij)
     and h (P^-1_jj - P^-1_ij) with w_i + w_j = c_k.
     At a fixed point the write-backs vanish and the step satisfies
     Eq. implicit_with_contact with the pair rows exactly.  The adjoint adds
     the pair rows to the KKT system (stick: z_i - z_j = 0; slip:
     (n - mu t).(z_i - z_j) = 0) with the friction term on the relative
     velocity, and the derivatives of n and beta with respect to x_i and x_j.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

TAKEOFF, STICK, SLIP = 0, 1, 2

# ----------------------------------------------------------------------------
# Rest-shape operators (readings R1, R2, R3)
# ----------------------------------------------------------------------------

# Vertex-to-edge matrix: F = X @ E @ Dm^-1 with X the 3x3 matrix of vertex positions.
_E = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])


def triangle_rest(rest, tris):
    """Per triangle: G = E Dm^-1 (3x2, so F = sum_a x_a G[a,:]) and rest area (R1)."""
    X0, X1, X2 = rest[tris[:, 0]], rest[tris[:, 1]], rest[tris[:, 2]]
    e1, e2 = X1 - X0, X2 - X0
    cr = np.cross(e1, e2)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    u = e1 / np.linalg.norm(e1, axis=1)[:, None]
    nrm = cr / np.linalg.norm(cr, axis=1)[:, None]
    w = np.cross(nrm, u)
    Dm = np.zeros((len(tris), 2, 2))
    Dm[:, 0, 0] = np.einsum("ij,ij->i", e1, u)
    Dm[:, 0, 1] = np.einsum("ij,ij->i", e2, u)
    Dm[:, 1, 0] = np.einsum("ij,ij->i", e1, w)
    Dm[:, 1, 1] = np.einsum("ij,ij->i", e2, w)
    G = np.einsum("ak,tkl->tal", _E, np.linalg.inv(Dm))
    return G, area


def cotan_laplacian(rest, tris, area):
    """Bending operator rows l_b (R2): (A_b x) = sum_j l_bj x_j, as a sparse m x m matrix.

    l_bj = c_bj / a_b for neighbours j, l_bb = -sum_j c_bj / a_b, where
    c_bj = (cot alpha + cot beta)/2 over the triangles sharing edge bj and a_b is
    one third of the rest area of the triangles around b.
    """
    m = rest.shape[0]
    rows, cols, vals = [], [], []
    for t in range(len(tris)):
        for k in range(3):
            o, i, j = tris[t, k], tris[t, (k + 1) % 3], tris[t, (k + 2) % 3]
            a = rest[i] - rest[o]
            b = rest[j] - rest[o]
            cot = np.dot(a, b) / np.linalg.norm(np.cross(a, b))
            rows += [i, j]
            cols += [j, i]
            vals += [0.5 * cot, 0.5 * cot]
    Wc = sp.coo_matrix((vals, (rows, cols)), shape=(m, m)).tocsr()
    abar = np.zeros(m)
    np.add.at(abar, tris.reshape(-1), np.repeat(area / 3.0, 3))
    deg = np.asarray(Wc.sum(axis=1)).ravel()
    Lap = (Wc - sp.diags(deg)).tocsr()
    Lb = sp.diags(1.0 / abar) @ Lap
    return Lb.tocsr(), abar


class Model:
    """Rest data, parameters and the prefactorised PD matrix of one cloth."""

    def __init__(self, rest_pos, tris, pins, obstacles, params):
        self.rest = np.asarray(rest_pos, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        self.m = self.rest.shape[0]
        self.pins = np.asarray(sorted(set(int(p) for p in pins)), dtype=np.int64)
        is_pin = np.zeros(self.m, bool)
        is_pin[self.pins] = True
        self.is_pin = is_pin
        self.free = np.nonzero(~is_pin)[0]
        self.obstacles = list(obstacles)
        self.params = params
        self.h = float(params.h)
        self.mu = float(params.mu)
        self.k_s = float(params.k_stretch)
        self.k_b = float(params.k_bend)
        self.g = np.asarray(params.gravity, dtype=np.float64)
        self.delta = float(params.contact_margin)
        self.self_thickness = float(getattr(params, "self_thickness", 0.0))
        self.compliance_mode = getattr(params, "contact_compliance", "rowsum")
        if self.compliance_mode not in ("rowsum", "diag_pinv", "diag_p", "mass"):
            raise ValueError(self.compliance_mode)

        self.G, self.area = triangle_rest(self.rest, self.tris)
        self.Lb, self.abar = cotan_laplacian(self.rest, self.tris, self.area)
        # R3: lumped mass
        self.mass = float(params.density) * self.abar
        # R2: target curvature magnitudes; a flat rest shape gives s_b = 0.
        q_rest = self.Lb @ self.rest
        s = np.linalg.norm(q_rest, axis=1)
        scale = (np.abs(self.Lb).sum(axis=1).A.ravel()
                 * np.max(np.linalg.norm(self.rest - self.rest.mean(0), axis=1)))
        s[s <= 1e-9 * scale] = 0.0
        self.s_b = s
        self.q_rest = q_rest
        self.w_t = self.k_s * self.area
        self.w_b = self.k_b * self.abar

        # Eq. pd_global: P = M + h^2 sum_i w_i A_i^T A_i.  Every A_i is (K_i kron I3),
        # so P = P_s kron I3 with a scalar m x m matrix P_s.
        self.L = self._stiffness_scalar()
        self.P = (sp.diags(self.mass) + self.h ** 2 * self.L).tocsr()
        self.Pff = self.P[self.free][:, self.free].tocsr()
        self._factor_banded()

    # --- assembly of sum_i w_i A_i^T A_i (scalar) ---
    def _stiffness_scalar(self):
        m = self.m
        T = len(self.tris)
        GG = np.einsum("tak,tbk->tab", self.G, self.G) * self.w_t[:, None, None]
        rows = np.repeat(self.tris, 3, axis=1).reshape(-1)
        cols = np.tile(self.tris, (1, 3)).reshape(-1)
        Ls = sp.coo_matrix((GG.reshape(-1), (rows, cols)), shape=(m, m)).tocsr()
        Lb = self.Lb
        Lbend = (Lb.T @ sp.diags(self.w_b) @ Lb).tocsr()
        del T
        return (Ls + Lbend).tocsr()

    def _factor_banded(self):
        """Banded Cholesky of P_ff in natural node order (upper band storage)."""
        A = self.Pff.tocoo()
        n = A.shape[0]
        bw = int(np.max(np.abs(A.row - A.col))) if A.nnz else 0
        ab = np.zeros((bw + 1, n))
        up = A.col >= A.row
        ab[bw + A.row[up] - A.col[up], A.col[up]] = A.data[up]
        self.band = bw
        self.chol = sla.cholesky_banded(ab, lower=False)

    def solve_P(self, rhs_f):
        """x = P_ff^-1 rhs on free nodes; rhs_f is (m_f,) or (m_f, k)."""
        return sla.cho_solve_banded((self.chol, False), rhs_f)

    # ------------------------------------------------------------------------
    # Local step (Sec. 3.1): projections of A_i x onto M_i
    # ------------------------------------------------------------------------
    def deformation_gradients(self, x):
        X = x[self.tris]                                 # (T, 3 vertices, 3 coords)
        return np.einsum("tac,tak->tck", X, self.G)      # F[t] = sum_a x_a G[a,:]

    def bending_vectors(self, x):
        return self.Lb @ x                               # (m, 3): A_b x

    def project(self, x):
        """Local step: p_t = polar factor of F_t (R1); p_b = s_b q/|q| (R2)."""
        F = self.deformation_gradients(x)
        R, S = polar(F)
        q = self.bending_vectors(x)
        pb = project_bending(q, self.s_b, self.q_rest)
        return R, pb, F, S, q

    def AtWp(self, R, pb):
        """sum_i w_i A_i^T p_i as an (m, 3) array."""
        out = np.zeros((self.m, 3))
        contrib = np.einsum("tck,tak->tac", R, self.G) * self.w_t[:, None, None]
        np.add.at(out, self.tris.reshape(-1), contrib.reshape(-1, 3))
        out += self.Lb.T @ (self.w_b[:, None] * pb)
        return out

    def energy_W(self, x):
        """Sum of the PD surrogate energies at their projections (Eq. pd_energy)."""
        R, pb, F, S, q = self.project(x)
        return self.surrogate_W(x, R, pb)

    def surrogate_W(self, x, R, pb):
        F = self.deformation_gradients(x)
        q = self.bending_vectors(x)
        ws = 0.5 * np.sum(self.w_t * np.sum((F - R) ** 2, axis=(1, 2)))
        wb = 0.5 * np.sum(self.w_b * np.sum((q - pb) ** 2, axis=1))
        return ws + wb

    def g_tilde(self, x, y, R, pb):
        """Surrogate objective of the local/global solver (Sec. 3.1)."""
        d = x - y
        return 0.5 / self.h ** 2 * np.sum(self.mass[:, None] * d * d) + self.surrogate_W(x, R, pb)

    # ------------------------------------------------------------------------
    # Contact detection (R4)
    # ------------------------------------------------------------------------
    def detect(self, x_n, v_n):
        """Contact list: (node, obstacle, normal n at x_n, beta = phi(x_n)/h)."""
        xp = x_n + self.h * v_n
        nodes, obs, normals, betas = [], [], [], []
        for j in self.free:
            best, best_o = np.inf, -1
            for o, ob in enumerate(self.obstacles):
                ph, _ = signed_distance(ob, xp[j])
                if ph < best:
                    best, best_o = ph, o
            if best_o >= 0 and best <= self.delta:
                ph0, n0 = signed_distance(self.obstacles[best_o], x_n[j])
                nodes.append(j)
                obs.append(best_o)
                normals.append(n0)
                betas.append(ph0 / self.h)
        return Contacts(np.array(nodes, dtype=np.int64), np.array(obs, dtype=np.int64),
                        np.array(normals).reshape(-1, 3), np.array(betas, dtype=np.float64))

    def detect_self(self, x_n, v_n):
        """Self-contact pairs (R13) from the predicted positions x_n + h v_n."""
        from scipy.spatial import cKDTree
        d_s = self.self_thickness
        xp = x_n + self.h * v_n
        if not hasattr(self, "_adjacent"):
            adj = set()
            for t in self.tris:
                for a in range(3):
                    for b in range(3):
                        if t[a] < t[b]:
                            adj.add((int(t[a]), int(t[b])))
            self._adjacent = adj
        pairs = sorted(cKDTree(xp).query_pairs(d_s + self.delta + 1e-12))
        ii, jj = [], []
        for a, b in pairs:
            i, j = (a, b) if a < b else (b, a)
            if (i, j) in self._adjacent or (self.is_pin[i] and self.is_pin[j]):
                continue
            # (nodes that coincide at x_n have no pair normal and are left out)
            if np.linalg.norm(xp[i] - xp[j]) <= d_s + self.delta and np.linalg.norm(x_n[i] - x_n[j]) > 0.0:
                ii.append(i)
                jj.append(j)
        ii = np.array(ii, dtype=np.int64)
        jj = np.array(jj, dtype=np.int64)
        d = x_n[ii] - x_n[jj]
        dist = np.linalg.norm(d, axis=1)
        normals = d / dist[:, None] if len(ii) else np.zeros((0, 3))
        wi, wj = self._pair_weights(ii, jj)
        return SelfContacts(ii, jj, normals.reshape(-1, 3), dist, (dist - d_s) / self.h, wi, wj)

    def _pair_weights(self, ii, jj):
        """Write-back weights of the pairs (R13): w_i : w_j = h (P^-1_ii - P^-1_ij) :
        h (P^-1_jj - P^-1_ij), scaled so that w_i + w_j is the pair's compliance
        c_k = sum_l |h (e_i - e_j)^T P^-1 (e_p - e_q)| (free nodes only: a pinned
        node has no row of P and its entries are 0)."""
        nf = len(self.free)
        pos = -np.ones(self.m, dtype=np.int64)
        pos[self.free] = np.arange(nf)
        npr = len(ii)
        D = np.zeros((nf, npr))                       # columns e_i - e_j (free rows)
        for a, (i, j) in enumerate(zip(ii, jj)):
            if pos[i] >= 0:
                D[pos[i], a] = 1.0
            if pos[j] >= 0:
                D[pos[j], a] = -1.0
        PD = self.solve_P(D) if npr else D            # P^-1 (e_i - e_j)
        W = self.h * (D.T @ PD)                       # pair coupling h (e_k)^T P^-1 (e_l)
        c = np.abs(W).sum(axis=1)
        wi, wj = np.zeros(npr), np.zeros(npr)
        for a, (i, j) in enumerate(zip(ii, jj)):
            # h P^-1 (e_i - e_j) restricted to rows i and -j
            ai = self.h * PD[pos[i], a] if pos[i] >= 0 else 0.0
            aj = -self.h * PD[pos[j], a] if pos[j] >= 0 else 0.0
            wi[a] = c[a] * ai / (ai + aj)
            wj[a] = c[a] * aj / (ai + aj)
        return wi, wj

    def couple_compliances(self, contacts, c, pairs):
        """With both obstacle contacts and self-contact pairs (R13), each side's
        Gershgorin bound also counts its coupling with the other kind:
        c_j += sum_k |h e_j^T P^-1 (e_p - e_q)| for an obstacle contact j and
        c_k += sum_j |h (e_p - e_q)^T P^-1 e_j| for a pair k (whose write-back
        weights are rescaled to the new c_k).  Returns the obstacle contacts' c."""
        nf = len(self.free)
        pos = -np.ones(self.m, dtype=np.int64)
        pos[self.free] = np.arange(nf)
        E = np.zeros((nf, len(contacts.nodes)))
        E[pos[contacts.nodes], np.arange(len(contacts.nodes))] = 1.0
        D = np.zeros((nf, len(pairs)))
        for a, (i, j) in enumerate(zip(pairs.i, pairs.j)):
            if pos[i] >= 0:
                D[pos[i], a] = 1.0
            if pos[j] >= 0:
                D[pos[j], a] = -1.0
        X = np.abs(self.h * (E.T @ self.solve_P(D)))   # |h e_j^T P^-1 (e_p - e_q)|
        c_new = pairs.c + X.sum(axis=0)
        scale = c_new / pairs.c
        pairs.wi = pairs.wi * scale
        pairs.wj = pairs.wj * scale
        pairs.c = c_new
        return c + X.sum(axis=1)

    def compliance(self, contacts):
        """c_j = h (P^-1 1_I)_j for the current contact set (R5), or the
        ablation choices h (P^-1)_jj, h / P_jj, h / m_j."""
        if len(contacts.nodes) == 0:
            return np.zeros(0)
        pos = np.searchsorted(self.free, contacts.nodes)
        if self.compliance_mode == "rowsum":
            ind = np.zeros(len(self.free))
            ind[pos] = 1.0
            return self.h * self.solve_P(ind)[pos]
        if self.compliance_mode == "diag_pinv":
            out = np.zeros(len(pos))
            for a, p in enumerate(pos):
                e = np.zeros(len(self.free))
                e[p] = 1.0
                out[a] = self.h * self.solve_P(e)[p]
            return out
        if self.compliance_mode == "diag_p":
            return self.h / self.Pff.diagonal()[pos]
        return self.h / self.mass[contacts.nodes]


class Contacts:
    def __init__(self, nodes, obs, normals, betas):
        self.nodes, self.obs, self.normals, self.betas = nodes, obs, normals, betas

    def __len__(self):
        return len(self.nodes)


class SelfContacts:
    """Node-node contact pairs (R13): nodes i < j, normal n from j to i at x_n,
    distance d = |x_i - x_j| at x_n, bias beta = (d - thickness)/h, and the
    write-back weights w_i, w_j with compliance c = w_i + w_j."""

    def __init__(self, i, j, normals, dist, betas, wi, wj):
        self.i, self.j, self.normals, self.dist, self.betas, self.wi, self.wj = i, j, normals, dist, betas, wi, wj
        self.c = wi + wj

    def __len__(self):
        return len(self.i)


# ----------------------------------------------------------------------------
# Projections
# ----------------------------------------------------------------------------

def polar(F):
    """Polar factor R and stretch S of 3x2 matrices F = R S (R1).

    S = sqrt(F^T F) in closed form for 2x2 SPD C = F^T F:
    S = (C + sqrt(det C) I) / sqrt(tr C + 2 sqrt(det C)), then R = F S^-1.
    sqrt(det C) is taken as |f_1 x f_2| (Lagrange's identity,
    det F^T F = |f_1 x f_2|^2 for the columns f_1, f_2 of F), which is exact
    for a triangle collapsed onto a line.  A collapsed triangle
    (det C <= 1e-30 (tr C)^2, see ``polar_degenerate``) has no unique polar
    factor; it gets the one of ``_polar_collapsed`` and S is left singular.
    """
    C = np.einsum("tck,tcl->tkl", F, F)
    cr = np.cross(F[:, :, 0], F[:, :, 1])
    sd = np.sqrt(np.einsum("tc,tc->t", cr, cr))
    tr = C[:, 0, 0] + C[:, 1, 1]
    t = np.sqrt(tr + 2.0 * sd)
    deg = polar_degenerate(F)
    S = np.zeros_like(C)
    ok = ~deg
    S[ok] = (C[ok] + sd[ok, None, None] * np.eye(2)) / t[ok, None, None]
    S[deg] = C[deg] / np.maximum(t[deg], 1e-300)[:, None, None]
    R = np.zeros_like(F)
    R[ok] = np.einsum("tck,tkl->tcl", F[ok], np.linalg.inv(S[ok]))
    for i in np.nonzero(deg)[0]:
        R[i] = _polar_collapsed(F[i])
    return R, S


def polar_degenerate(F):
    """Reading R1, degenerate case: det(F^T F) <= 1e-30 (tr F^T F)^2, i.e. the
    smaller singular value of F is at most ~1e-15 of the larger one."""
    cr = np.cross(F[:, :, 0], F[:, :, 1])
    det = np.einsum("tc,tc->t", cr, cr)
    tr = np.einsum("tck,tck->t", F, F)
    return det <= 1e-30 * tr * tr


def _polar_collapsed(F):
    """A polar factor of a 3x2 F of rank <= 1 (reading R1, degenerate case), from
    the singular vectors of F with the missing left vector chosen by a fixed rule:
    v1 = the eigenvector of C = F^T F of its larger eigenvalue, v2 = v1 rotated
    by +90 degrees; u1 = F v1 / |F v1|; u2 = normalize(u1 x e_a) with e_a the
    first coordinate axis (x, y, z order) with |u1_a| <= 0.6 (one exists since
    1/sqrt(3) < 0.6; the choice only changes where a component crosses 0.6, far
    from the axis-aligned collapses whose other components are rounding noise);
    R = u1 v1^T + u2 v2^T.  F = 0 gives R = [e_x, e_y]."""
    C = F.T @ F
    tr = C[0, 0] + C[1, 1]
    if tr == 0.0:
        return np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    d = 0.5 * (C[0, 0] - C[1, 1])
    r = np.hypot(d, C[0, 1])
    v1 = np.array([d + r, C[0, 1]]) if d >= 0.0 else np.array([C[0, 1], r - d])
    v1 = v1 / np.linalg.norm(v1)
    v2 = np.array([-v1[1], v1[0]])
    w1 = F @ v1
    u1 = w1 / np.linalg.norm(w1)
    a = int(np.nonzero(np.abs(u1) <= 0.6)[0][0])
    e = np.zeros(3)
    e[a] = 1.0
    u2 = np.cross(u1, e)
    u2 = u2 / np.linalg.norm(u2)
    return np.outer(u1, v1) + np.outer(u2, v2)


def project_bending(q, s_b, q_rest):
    """p_b = s_b q/|q| where s_b > 0, 0 where s_b = 0; q_rest if |q| collapses (R2)."""
    nq = np.linalg.norm(q, axis=1)
    pb = np.zeros_like(q)
    on = s_b > 0
    ok = on & (nq > 1e-14 * s_b)
    pb[ok] = (s_b[ok] / nq[ok])[:, None] * q[ok]
    tie = on & ~ok
    pb[tie] = q_rest[tie]
    return pb


def polar_derivative(R, S, dF):
    """dR for F = R S perturbed by dF (3x2): dR = R Om + (I - R R^T) dF S^-1 with
    Om = w [[0,-1],[1,0]], w = ((R^T dF)_21 - (R^T dF)_12) / tr S.  (Not defined
    for a collapsed triangle; ``hessian_W`` takes dR = 0 there, reading R1.)"""
    RtdF = R.T @ dF
    w = (RtdF[1, 0] - RtdF[0, 1]) / np.trace(S)
    Om = np.array([[0.0, -w], [w, 0.0]])
    return R @ Om + (np.eye(3) - R @ R.T) @ dF @ np.linalg.inv(S)


# ----------------------------------------------------------------------------
# Obstacles (R4)
# ----------------------------------------------------------------------------

def _closest_on_triangle(x, P):
    """Closest point of triangle P (3 x 3, rows = vertices) to x, and its feature:
    ("face",), ("edge", i, j) or ("vertex", i) with local vertex indices.  The
    projection onto the triangle's plane is kept if its barycentric coordinates
    are all >= 0; otherwise the closest point is the nearest of the three edge
    segments' closest points (first edge on ties)."""
    A, B, C = P
    nrm = np.cross(B - A, C - A)
    nrm = nrm / np.linalg.norm(nrm)
    p = x - np.dot(x - A, nrm) * nrm
    v0, v1, v2 = B - A, C - A, p - A
    d00, d01, d11 = np.dot(v0, v0), np.dot(v0, v1), np.dot(v1, v1)
    d20, d21 = np.dot(v2, v0), np.dot(v2, v1)
    den = d00 * d11 - d01 * d01
    bv = (d11 * d20 - d01 * d21) / den
    bw = (d00 * d21 - d01 * d20) / den
    if bv >= 0.0 and bw >= 0.0 and 1.0 - bv - bw >= 0.0:
        return p, ("face",)
    best = None
    for i, j in ((0, 1), (1, 2), (2, 0)):
        Q0, Q1 = P[i], P[j]
        t = np.clip(np.dot(x - Q0, Q1 - Q0) / np.dot(Q1 - Q0, Q1 - Q0), 0.0, 1.0)
        c = Q0 + t * (Q1 - Q0)
        d = np.linalg.norm(x - c)
        feat = ("vertex", i) if t == 0.0 else (("vertex", j) if t == 1.0 else ("edge", i, j))
        if best is None or d < best[0]:
            best = (d, c, feat)
    return best[1], best[2]


# Distances within MESH_TIE (relative, plus MESH_TIE_ABS) of the smallest count as
# ties, which the lowest face index wins; closer than MESH_ON_SURFACE (metres) a
# point is on the surface and takes as normal the pseudo-normal of the feature its
# closest point lies on to within MESH_SNAP metres (a vertex, else an edge, else
# the face).
MESH_TIE = 1e-9
MESH_TIE_ABS = 1e-14
MESH_ON_SURFACE = 1e-12
MESH_SNAP = 1e-9


def _snap_feature(P, c):
    """The feature of triangle P (rows = vertices) that the point c on it lies on
    to within MESH_SNAP: ("vertex", k) for the first vertex, else ("edge", k, k+1)
    for the first edge AB, BC, CA, else ("face",) (local indices)."""
    for k in range(3):
        if np.linalg.norm(c - P[k]) <= MESH_SNAP:
            return ("vertex", k)
    for k in range(3):
        a, b = P[k], P[(k + 1) % 3]
        t = np.clip(np.dot(c - a, b - a) / np.dot(b - a, b - a), 0.0, 1.0)
        if np.linalg.norm(c - (a + t * (b - a))) <= MESH_SNAP:
            return ("edge", k, (k + 1) % 3)
    return ("face",)


def _mesh_closest(ob, x):
    """Closest point of a closed triangle mesh to x: (point, distance, feature in
    mesh vertex indices, face index).  Among faces whose distance is within
    MESH_TIE of the smallest, the lowest face index wins, so that points
    equidistant from several faces (symmetric configurations) are not decided
    by rounding."""
    V = np.asarray(ob.vertices, dtype=np.float64)
    F = np.asarray(ob.triangles, dtype=np.int64)
    cand = []
    for f in range(len(F)):
        c, feat = _closest_on_triangle(x, V[F[f]])
        cand.append((c, float(np.linalg.norm(x - c)), feat))
    dmin = min(d for _, d, _ in cand)
    for f, (c, d, feat) in enumerate(cand):
        if d <= dmin * (1.0 + MESH_TIE) + MESH_TIE_ABS:
            if feat[0] == "edge":
                feat = ("edge", int(F[f][feat[1]]), int(F[f][feat[2]]))
            elif feat[0] == "vertex":
                feat = ("vertex", int(F[f][feat[1]]))
            return c, d, feat, f


def _mesh_pseudo_normal(ob, feat, face):
    """Angle-weighted pseudo-normal of a mesh feature (its sign test tells inside
    from outside): the face normal; the sum of the two incident face normals for
    an edge; the sum of incident face normals weighted by their angle at a vertex."""
    V = np.asarray(ob.vertices, dtype=np.float64)
    F = np.asarray(ob.triangles, dtype=np.int64)

    def fn(f):
        a, b, c = V[F[f]]
        n = np.cross(b - a, c - a)
        return n / np.linalg.norm(n)
    if feat[0] == "face":
        return fn(face)
    if feat[0] == "edge":
        i, j = feat[1], feat[2]
        fs = [f for f in range(len(F)) if i in F[f] and j in F[f]]
        return sum(fn(f) for f in fs)
    i = feat[1]
    out = np.zeros(3)
    for f in range(len(F)):
        if i in F[f]:
            k = list(F[f]).index(i)
            p, q = V[F[f][(k + 1) % 3]] - V[i], V[F[f][(k + 2) % 3]] - V[i]
            ang = np.arccos(np.clip(np.dot(p, q) / (np.linalg.norm(p) * np.linalg.norm(q)), -1.0, 1.0))
            out += ang * fn(f)
    return out


def signed_distance(ob, x):
    """(phi, grad phi) of an obstacle at point x."""
    if ob.kind == "mesh":
        # |x - c| to the closest point c, signed by the pseudo-normal N of c's
        # feature; grad phi = s (x - c)/|x - c|.  On the surface (|x - c| below
        # MESH_ON_SURFACE, where a stick or slip step leaves a node and (x - c) is
        # rounding) the normal is N/|N|.
        c, d, feat, face = _mesh_closest(ob, x)
        N = _mesh_pseudo_normal(ob, feat, face)
        s = 1.0 if np.dot(x - c, N) >= 0.0 else -1.0
        if d < MESH_ON_SURFACE:
            Fi = np.asarray(ob.triangles, dtype=np.int64)[face]
            sf = _snap_feature(np.asarray(ob.vertices, dtype=np.float64)[Fi], c)
            sf = sf if sf[0] == "face" else (sf[0],) + tuple(int(Fi[k]) for k in sf[1:])
            Ns = _mesh_pseudo_normal(ob, sf, face)
            return float(s * d), Ns / np.linalg.norm(Ns)
        return float(s * d), s * (x - c) / d
    if ob.kind == "plane":
        n = np.asarray(ob.normal, dtype=np.float64)
        return float(np.dot(n, x) - ob.offset), n.copy()
    if ob.kind == "sphere":
        d = x - np.asarray(ob.center, dtype=np.float64)
        r = np.linalg.norm(d)
        return float(r - ob.radius), d / r
    if ob.kind == "capsule":
        a = np.asarray(ob.a, dtype=np.float64)
        b = np.asarray(ob.b, dtype=np.float64)
        ab = b - a
        t = np.clip(np.dot(x - a, ab) / np.dot(ab, ab), 0.0, 1.0)
        d = x - (a + t * ab)
        r = np.linalg.norm(d)
        return float(r - ob.radius), d / r
    raise ValueError(ob.kind)


def normal_jacobian(ob, x):
    """d n / d x for the obstacle normal taken at x (3x3); zero for planes, in
    the face region of a mesh and on a mesh's surface; s (I - u u^T - e e^T)/r on a mesh edge (e its unit
    direction), s (I - u u^T)/r at a mesh vertex, u = (x - c)/r, r = |x - c|."""
    if ob.kind == "plane":
        return np.zeros((3, 3))
    if ob.kind == "mesh":
        c, r, feat, face = _mesh_closest(ob, x)
        if feat[0] == "face" or r < MESH_ON_SURFACE:
            return np.zeros((3, 3))
        s = 1.0 if np.dot(x - c, _mesh_pseudo_normal(ob, feat, face)) >= 0.0 else -1.0
        u = (x - c) / r
        J = np.eye(3) - np.outer(u, u)
        if feat[0] == "edge":
            V = np.asarray(ob.vertices, dtype=np.float64)
            e = V[feat[2]] - V[feat[1]]
            e = e / np.linalg.norm(e)
            J = J - np.outer(e, e)
        return s * J / r
    if ob.kind == "sphere":
        d = x - np.asarray(ob.center, dtype=np.float64)
        r = np.linalg.norm(d)
        n = d / r
        return (np.eye(3) - np.outer(n, n)) / r
    if ob.kind == "capsule":
        a = np.asarray(ob.a, dtype=np.float64)
        b = np.asarray(ob.b, dtype=np.float64)
        ab = b - a
        t = np.dot(x - a, ab) / np.dot(ab, ab)
        if t <= 0.0 or t >= 1.0:
            c = a if t <= 0.0 else b
            d = x - c
            r = np.linalg.norm(d)
            n = d / r
            return (np.eye(3) - np.outer(n, n)) / r
        e = ab / np.linalg.norm(ab)
        d = x - (a + t * ab)
        r = np.linalg.norm(d)
        n = d / r
        return (np.eye(3) - np.outer(n, n) - np.outer(e, e)) / r
    raise ValueError(ob.kind)


# ----------------------------------------------------------------------------
# Per-node Signorini-Coulomb solve (Eq. contact_all), closed form (R5)
# ----------------------------------------------------------------------------

def signorini_coulomb(vt, n, beta, mu, c):
    """Solve v = vt + c f with (f, u) satisfying Eq. contact_1-3 in world frame.

    u_N = n.v + beta, u_T = v - (n.v) n.  Returns (f, v, case)."""
    vn = float(np.dot(n, vt))
    uN = vn + beta
    if uN >= 0.0:                                     # take off: r = 0, u_N > 0
        return np.zeros(3), vt.copy(), TAKEOFF
    uT = vt - vn * n
    nt = float(np.linalg.norm(uT))
    if nt <= mu * (-uN):                              # stick: u = 0, |r_T| <= mu r_N
        v = -beta * n
        return (v - vt) / c, v, STICK
    fN = -uN / c                                      # slip: u_N = 0, |r_T| = mu r_N
    f = fN * n - (mu * fN / nt) * uT
    return f, vt + c * f, SLIP


# ----------------------------------------------------------------------------
# One time step (Sec. 3.1-3.2)
# ----------------------------------------------------------------------------

class StepRecord:
    """What the adjoint needs from a converged forward step."""

    def __init__(self, x_n, v_n, x_np1, v_np1, contacts, forces, cases, c, iters, pairs=None, pair_forces=None,
                 pair_cases=None):
        self.x_n, self.v_n, self.x_np1, self.v_np1 = x_n, v_n, x_np1, v_np1
        self.contacts, self.forces, self.cases, self.c, self.iters = contacts, forces, cases, c, iters
        # self-contact pairs (R13): SelfContacts, their impulses r (on node i) and cases
        self.pairs = pairs if pairs is not None else SelfContacts(*([np.zeros(0, np.int64)] * 2),
                                                                  np.zeros((0, 3)), *([np.zeros(0)] * 4))
        self.pair_forces = pair_forces if pair_forces is not None else np.zeros((0, 3))
        self.pair_cases = pair_cases if pair_cases is not None else np.zeros(0, dtype=np.int64)


def step(model: Model, x_n, v_n, n_iters=None, tol=None, max_iters=100000, trace=None):
    """One PD time step with dry frictional contact.

    Fixed-iteration mode (n_iters): exactly that many local/global/contact
    iterations (the method as run for timing and parity).  Tolerance mode
    (tol): iterate until the max-norm change of v is below tol * max(|v|, 1e-3).
    ``trace`` (a list) receives g~ after every local and every global step.
    """
    h = model.h
    free = model.free
    x_n = np.asarray(x_n, dtype=np.float64)
    v_n = np.asarray(v_n, dtype=np.float64).copy()
    v_n[model.pins] = 0.0
    # Eq. implicit_energy: y = x_n + h v_n + h^2 M^-1 f_ext, f_ext = M g (R3)
    y = x_n + h * v_n + h * h * model.g[None, :]
    # b^(p) = (b(p) - P x_n)/h with b(p) = M y + h^2 sum w A^T p and P = M + h^2 sum w A^T A
    # (Eq. pd_global, pd_velocity), expanded so that no O(h^2 |L x|) terms cancel:
    #   b^(p) = M (y - x_n)/h + h sum_i w_i A_i^T (p_i - A_i x_n).
    Mdy = model.mass[:, None] * (y - x_n) / h
    F_n = model.deformation_gradients(x_n)
    q_n = model.bending_vectors(x_n)
    contacts = model.detect(x_n, v_n)                  # J_n from (x_n, v_n), Eq. implicit_with_contact
    c = model.compliance(contacts)
    nc = len(contacts)
    f = np.zeros((nc, 3))
    cases = np.zeros(nc, dtype=np.int64)
    pairs = model.detect_self(x_n, v_n) if model.self_thickness > 0.0 else None   # R13
    npr = len(pairs) if pairs is not None else 0
    if npr and nc:
        c = model.couple_compliances(contacts, c, pairs)
    fp = np.zeros((npr, 3))
    pcases = np.zeros(npr, dtype=np.int64)
    v = v_n.copy()
    if n_iters is None and tol is None:
        n_iters = model.params.n_pd_iters
    limit = n_iters if n_iters is not None else max_iters
    k = 0
    mass_split = model.compliance_mode == "mass"
    while k < limit:
        x = x_n + h * v
        R, pb, F_k, _, q_k = model.project(x)                      # local step
        if trace is not None:
            trace.append(model.g_tilde(x, y, R, pb))
        if mass_split:
            # Eq. ly_et_al_govrningEq as printed: M v_half = b - (P - M) v^k + h J^T r,
            # with b - (P - M) v^k = M (y - x_n)/h + h sum_i w_i A_i^T (p_i - A_i x^k)
            bhat = Mdy + h * model.AtWp(R - F_k, pb - q_k)
        else:
            bhat = Mdy + h * model.AtWp(R - F_n, pb - q_n)         # Eq. pd_global / pd_velocity
        rhs = bhat.copy()
        if nc:
            rhs[contacts.nodes] += h * f                           # Eq. pd_velocity_with_contact
        if npr:                                                    # pair rows: +r on i, -r on j
            np.add.at(rhs, pairs.i, h * fp)
            np.add.at(rhs, pairs.j, -h * fp)
        v_half = np.zeros_like(v)
        if mass_split:
            v_half[free] = rhs[free] / model.mass[free][:, None]   # global step of the mass splitting
        else:
            v_half[free] = model.solve_P(rhs[free])                # global step
        if trace is not None:
            trace.append(model.g_tilde(x_n + h * v_half, y, R, pb))
        v_new = v_half
        f_new = np.zeros_like(f)
        if npr:
            v_new = v_half.copy()
        for a in range(nc):                                        # per-node contact solve
            j = contacts.nodes[a]
            vt = v_half[j] - c[a] * f[a]
            f_new[a], v_new[j], cases[a] = signorini_coulomb(
                vt, contacts.normals[a], contacts.betas[a], model.mu, c[a])
        fp_new = np.zeros_like(fp)
        for a in range(npr):                                       # pair solves from v_half (R13)
            i, j = pairs.i[a], pairs.j[a]
            ut = v_half[i] - v_half[j] - pairs.c[a] * fp[a]
            fp_new[a], _, pcases[a] = signorini_coulomb(ut, pairs.normals[a], pairs.betas[a], model.mu, pairs.c[a])
            dr = fp_new[a] - fp[a]
            v_new[i] += pairs.wi[a] * dr
            v_new[j] -= pairs.wj[a] * dr
        dv = np.max(np.abs(v_new - v)) if v.size else 0.0
        v, f, fp = v_new, f_new, fp_new
        k += 1
        if tol is not None and dv <= tol * max(np.max(np.abs(v)), 1e-3):
            break
    x_np1 = x_n + h * v
    return x_np1, v, StepRecord(x_n, v_n, x_np1, v, contacts, f, cases, c, k, pairs, fp, pcases)


def rollout(model: Model, x0, v0, n_steps, n_iters=None, tol=None):
    """Run n_steps; returns (xs, vs, records) with xs[0] = x0."""
    xs, vs, recs = [np.asarray(x0, dtype=np.float64)], [np.asarray(v0, dtype=np.float64)], []
    for _ in range(n_steps):
        x1, v1, rec = step(model, xs[-1], vs[-1], n_iters=n_iters, tol=tol)
        xs.append(x1)
        vs.append(v1)
        recs.append(rec)
    return xs, vs, recs


# ----------------------------------------------------------------------------
# Adjoint (Sec. 4), reading R7
# ----------------------------------------------------------------------------

def _dof(nodes):
    nodes = np.asarray(nodes)
    return (3 * nodes[:, None] + np.arange(3)[None, :]).reshape(-1)


def hessian_W(model: Model, x):
    """grad^2 W(x) = sum_i w_i A_i^T (I - d p_i*/d(A_i x)) A_i as a 3m x 3m matrix (Sec. 4.1)."""
    m = model.m
    R, pb, F, S, q = model.project(x)
    rows, cols, vals = [], [], []
    T = len(model.tris)
    # stretch: vec(F) index (c, k) -> 3*k + c; A_t[(c,k), (a,c')] = G[a,k] delta_cc'
    deg = polar_degenerate(F)
    for t in range(T):
        A = np.zeros((6, 9))
        for a in range(3):
            for k in range(2):
                for cc in range(3):
                    A[3 * k + cc, 3 * a + cc] = model.G[t, a, k]
        Jp = np.zeros((6, 6))
        for e in range(6 if not deg[t] else 0):   # collapsed: projection taken as locally constant (R1)
            dF = np.zeros((3, 2))
            dF[e % 3, e // 3] = 1.0
            dR = polar_derivative(R[t], S[t], dF)
            Jp[:, e] = dR.T.reshape(-1)          # column-major vec: index 3*k + c
        Ht = model.w_t[t] * A.T @ (np.eye(6) - Jp) @ A
        d = _dof(model.tris[t])
        rows.append(np.repeat(d, 9))
        cols.append(np.tile(d, 9))
        vals.append(Ht.reshape(-1))
    # bending: A_b = l_b kron I3
    Lb = model.Lb.tocsr()
    for b in range(m):
        lo, hi = Lb.indptr[b], Lb.indptr[b + 1]
        nb = Lb.indices[lo:hi]
        lv = Lb.data[lo:hi]
        if model.s_b[b] > 0:
            nq = np.linalg.norm(q[b])
            qh = q[b] / nq
            Dp = model.s_b[b] * (np.eye(3) - np.outer(qh, qh)) / nq
        else:
            Dp = np.zeros((3, 3))
        K = np.eye(3) - Dp
        blk = model.w_b[b] * np.einsum("i,j,cd->icjd", lv, lv, K).reshape(3 * len(nb), 3 * len(nb))
        d = _dof(nb)
        rows.append(np.repeat(d, len(d)))
        cols.append(np.tile(d, len(d)))
        vals.append(blk.reshape(-1))
    Hm = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(3 * m, 3 * m)).tocsr()
    return Hm, (R, pb, F, S, q)


def adjoint_step(model: Model, rec: StepRecord, gx, gv, hess=None, permc_spec=None):
    """Back-propagate (dL/dx_{n+1}, dL/dv_{n+1}) through one converged step.

    ``hess``, if given, is ``hessian_W(model, rec.x_np1)`` computed beforehand
    (e.g. for many steps in parallel); the result is the same.  ``permc_spec``
    picks the column ordering of the sparse LU (scipy's default if None); two
    orderings give the same solution up to rounding, and their difference shows
    how much rounding the KKT system amplifies.

    Returns (dL/dx_n, dL/dv_n, dL/d[k_stretch, k_bend, mu], z, eta).

    Unknowns of the linearised step: dv (free DOFs) and the contact multipliers
    (stick: the 3D force; slip: the normal force; take-off: none).  Its
    transpose gives the adjoint system
        H z + B eta = g,   C^T z = 0,   g = dL/dv_{n+1} + h dL/dx_{n+1},
    H = M + h^2 grad^2 W(x_{n+1}) + sum_slip h mu f_N b b^T / |u_T|
    (Eq. adjoint_v with the contact term of Eq. ppr_adjoint), and
    dL/dv_n = M z (Eq. adjoint_v), dL/dx_n = dL/dx_{n+1} - h grad^2 W z - contact terms.
    """
    h, mu = model.h, model.mu
    m = model.m
    free = model.free
    x1, v1 = rec.x_np1, rec.v_np1
    gx = np.asarray(gx, dtype=np.float64)
    gv = np.asarray(gv, dtype=np.float64)
    g = gv + h * gx
    Hw, (R, pb, F, S, q) = hessian_W(model, x1) if hess is None else hess
    Mfull = sp.diags(np.repeat(model.mass, 3))
    fd = _dof(free)
    H = (Mfull + h * h * Hw)[fd][:, fd].tolil()
    pos_of = -np.ones(m, dtype=np.int64)
    pos_of[free] = np.arange(len(free))
    Bcols, Ccols = [], []
    ctr = rec.contacts
    tdirs = {}
    for a in range(len(ctr)):
        j = ctr.nodes[a]
        nrm = ctr.normals[a]
        base = 3 * pos_of[j]
        if rec.cases[a] == STICK:
            for e in range(3):
                col = np.zeros(3)
                col[e] = 1.0
                Bcols.append([(base, col)])
                Ccols.append([(base, col)])
        elif rec.cases[a] == SLIP:
            uT = v1[j] - np.dot(nrm, v1[j]) * nrm
            nt = np.linalg.norm(uT)
            th = uT / nt
            bh = np.cross(nrm, th)
            fN = float(np.dot(rec.forces[a], nrm))
            blk = h * mu * fN / nt * np.outer(bh, bh)
            for r_ in range(3):
                for c_ in range(3):
                    H[base + r_, base + c_] += blk[r_, c_]
            Bcols.append([(base, nrm.copy())])
            Ccols.append([(base, nrm - mu * th)])
            tdirs[a] = (th, nt, fN)
    # self-contact pairs (R13): rows on the relative velocity, +1 block at i, -1 at j
    prs = rec.pairs
    pdirs = {}
    for a in range(len(prs)):
        i, j = prs.i[a], prs.j[a]
        nrm = prs.normals[a]
        ends = [(3 * pos_of[i], 1.0)] if pos_of[i] >= 0 else []
        if pos_of[j] >= 0:
            ends.append((3 * pos_of[j], -1.0))
        if rec.pair_cases[a] == STICK:
            for e in range(3):
                col = np.zeros(3)
                col[e] = 1.0
                Bcols.append([(b, sg * col) for b, sg in ends])
                Ccols.append([(b, sg * col) for b, sg in ends])
        elif rec.pair_cases[a] == SLIP:
            u = v1[i] - v1[j]
            uT = u - np.dot(nrm, u) * nrm
            nt = np.linalg.norm(uT)
            th = uT / nt
            bh = np.cross(nrm, th)
            fN = float(np.dot(rec.pair_forces[a], nrm))
            blk = h * mu * fN / nt * np.outer(bh, bh)
            for b1, s1 in ends:
                for b2, s2 in ends:
                    for r_ in range(3):
                        for c_ in range(3):
                            H[b1 + r_, b2 + c_] += s1 * s2 * blk[r_, c_]
            Bcols.append([(b, sg * nrm) for b, sg in ends])
            Ccols.append([(b, sg * (nrm - mu * th)) for b, sg in ends])
            pdirs[a] = (th, nt, fN)
    H = H.tocsr()
    nf3 = 3 * len(free)
    nk = len(Bcols)
    Bm = sp.lil_matrix((nf3, nk))
    Cm = sp.lil_matrix((nf3, nk))
    for col, (bblocks, cblocks) in enumerate(zip(Bcols, Ccols)):
        for base, bv in bblocks:
            for e in range(3):
                Bm[base + e, col] += bv[e]
        for base, cv in cblocks:
            for e in range(3):
                Cm[base + e, col] += cv[e]
    K = sp.bmat([[H, Bm.tocsr()], [Cm.tocsr().T, None]], format="csc")
    rhs = np.concatenate([g[free].reshape(-1), np.zeros(nk)])
    sol = spla.spsolve(K, rhs, permc_spec=permc_spec) if nk or nf3 else rhs
    sol = np.atleast_1d(sol)
    z = np.zeros((m, 3))
    z[free] = sol[:nf3].reshape(-1, 3)
    eta = sol[nf3:]

    # dL/dv_n = M z   (pinned velocities are fixed, their gradient is 0)
    dv_n = model.mass[:, None] * z
    dv_n[model.pins] = 0.0
    # dL/dx_n = dL/dx_{n+1} - (dF/dx_n)^T z - (dG/dx_n)^T eta, dF/dx_n = h grad^2 W
    dx_n = gx - h * (Hw @ z.reshape(-1)).reshape(m, 3)
    # parameters: dF/dk_s = h sum_t area_t A_t^T (A_t x - p_t), similarly k_b;
    # dF/dmu = h sum_slip f_N t (slip force f = f_N (n - mu t)).
    Fz = model.deformation_gradients(z)
    qz = model.bending_vectors(z)
    dks = -h * np.sum(model.area * np.sum(Fz * (F - R), axis=(1, 2)))
    dkb = -h * np.sum(model.abar * np.sum(qz * (q - pb), axis=1))
    dmu = 0.0
    col = 0
    for a in range(len(ctr)):
        j = ctr.nodes[a]
        ob = model.obstacles[ctr.obs[a]]
        nrm = ctr.normals[a]
        Dn = normal_jacobian(ob, rec.x_n[j])
        beta = ctr.betas[a]
        if rec.cases[a] == STICK:
            psi = eta[col:col + 3]
            col += 3
            # G_j = v_j + beta n:  dG/dx_n = beta Dn + n n^T / h
            dx_n[j] -= beta * Dn.T @ psi + nrm * np.dot(nrm, psi) / h
        elif rec.cases[a] == SLIP:
            psi = eta[col]
            col += 1
            th, nt, fN = tdirs[a]
            vj = v1[j]
            dmu += -h * fN * np.dot(th, z[j])
            # dt/dx_n through the normal: t = Pi v/|Pi v|, Pi = I - n n^T
            dPiv = -(np.dot(nrm, vj) * np.eye(3) + np.outer(nrm, vj)) @ Dn
            Dt = (np.eye(3) - np.outer(th, th)) @ dPiv / nt
            # F_j contains -h f_N (n - mu t): contributes +h f_N (Dn - mu Dt)^T z_j
            dx_n[j] += h * fN * (Dn - mu * Dt).T @ z[j]
            # G_j = n.v_j + beta: dG/dx_n = Dn^T v_j + n / h
            dx_n[j] -= (Dn.T @ vj + nrm / h) * psi
    # self-contact pairs (R13): n = (x_i - x_j)/d and beta = (d - thickness)/h depend on
    # x_i (derivatives Dn = (I - n n^T)/d and n/h) and on x_j (their negatives)
    for a in range(len(prs)):
        i, j = prs.i[a], prs.j[a]
        nrm = prs.normals[a]
        Dn = (np.eye(3) - np.outer(nrm, nrm)) / prs.dist[a]
        beta = prs.betas[a]
        if rec.pair_cases[a] == STICK:
            psi = eta[col:col + 3]
            col += 3
            # G = v_i - v_j + beta n:  dG/dx_i = beta Dn + n n^T / h = -dG/dx_j
            gi = beta * Dn.T @ psi + nrm * np.dot(nrm, psi) / h
            dx_n[i] -= gi
            dx_n[j] += gi
        elif rec.pair_cases[a] == SLIP:
            psi = eta[col]
            col += 1
            th, nt, fN = pdirs[a]
            u = v1[i] - v1[j]
            dz = z[i] - z[j]
            dmu += -h * fN * np.dot(th, dz)
            dPiu = -(np.dot(nrm, u) * np.eye(3) + np.outer(nrm, u)) @ Dn
            Dt = (np.eye(3) - np.outer(th, th)) @ dPiu / nt
            # F_i holds -h f_N (n - mu t) and F_j its negative
            gi = h * fN * (Dn - mu * Dt).T @ dz
            dx_n[i] += gi
            dx_n[j] -= gi
            # G = n.(v_i - v_j) + beta: dG/dx_i = Dn^T u + n / h = -dG/dx_j
            gi = (Dn.T @ u + nrm / h) * psi
            dx_n[i] -= gi
            dx_n[j] += gi
    return dx_n, dv_n, np.array([dks, dkb, dmu]), z, eta


def rollout_gradient(model: Model, records, dL_dx_final, dL_dv_final=None, dL_dtraj_x=None, hessians=None,
                     permc_spec=None):
    """Reverse pass over a rollout: returns (dL/dx0, dL/dv0, dL/d[k_s, k_b, mu]).
    ``hessians[n]``, if given, is hessian_W at records[n].x_np1; ``permc_spec`` as
    for adjoint_step."""
    gx = np.asarray(dL_dx_final, dtype=np.float64).copy()
    gv = np.zeros_like(gx) if dL_dv_final is None else np.asarray(dL_dv_final, dtype=np.float64).copy()
    dth = np.zeros(3)
    N = len(records)
    for n in range(N - 1, -1, -1):
        if dL_dtraj_x is not None:
            gx = gx + dL_dtraj_x[n + 1]
        gx, gv, d, _, _ = adjoint_step(model, records[n], gx, gv, None if hessians is None else hessians[n],
                                       permc_spec)
        dth += d
    if dL_dtraj_x is not None:
        gx = gx + dL_dtraj_x[0]
    return gx, gv, dth


def model_from_scene(scene, **overrides):
    """Convenience: build a Model from a scenes.Scene, optionally overriding parameters."""
    import dataclasses
    prm = dataclasses.replace(scene.params, **overrides) if overrides else scene.params
    return Model(scene.rest_pos, scene.tris, scene.pins, scene.obstacles, prm)
