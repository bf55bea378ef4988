"""The paper's seven main steps, plainly -- oracle, test only.

Eq. (1): eliminating E from [[A, D], [D^T, 0]] [E; lambda] = [f; 0] gives
    K lambda = g,  K = sum_i D_i^T A_i^{-1} D_i,  g = sum_i D_i^T A_i^{-1} f_i,
and then E_i = A_i^{-1} (f_i - D_i lambda).

  step 1  dense domain matrices K_D^(i) = D_i^T A_i^{-1} D_i  (A_i^{-1} by
          SciPy sparse LU on the columns of D_i, or dense inverse if asked)
  step 2  assemble K from the K_D^(i)
  step 3  block nested dissection of the interface blocks (ordering.py)
  step 4  block symbolic factorisation by the elimination game on blocks
  step 5  Algorithm 1, block LDL^T with restricted Bunch-Kaufman pivots,
          read as (the printed indices are inconsistent):
            P_j K_jj P_j^T = L_jj D_jj L_jj^T
            X_ij = K_ij P_j^T L_jj^{-T}     (triangular solve, = L_ij D_jj)
            L_ij = X_ij D_jj^{-1}           (the work variable W_ij)
            K_ik <- K_ik - L_ij X_kj^T      for every pair i >= k > j
          with plain transposes (K is complex symmetric).
  step 6  forward / diagonal / backward substitution for lambda
  step 7  recover E_i and take each edge from its owner copy.

A second, independent route to the same solution (solve_primal_schur): the
classical primal substructuring of the same decomposed operators, with one
unknown per interface edge instead of multipliers -- eliminate every
subdomain's interior, sum the interface Schur complements (the +-alpha
interface terms cancel there), solve, recover the interiors.

Parity pins (tests/test_oracle_d3m.py): E equals the undecomposed global
solution, for several interface coefficients alpha; K equals brute-force
D^T A^{-1} D with dense inverses; the block LDL^T reproduces K and solves it
like numpy.linalg.solve; the primal Schur route equals both.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import bk, decomp, fem, ordering


def domain_matrix(A, Dc, which=None, lu=None):
    """Step 1 for one subdomain: K_D = D_i^T A_i^{-1} D_i with D_i restricted
    to its nonzero columns (Dc, dense); with `which`, only those columns of
    K_D (A_i^{-1} applied to those columns of Dc).  A_i^{-1} by SciPy sparse
    LU (given in `lu`, or computed here)."""
    lu = spla.splu(A.tocsc()) if lu is None else lu
    B = Dc if which is None else Dc[:, which]
    return Dc.T @ lu.solve(np.asarray(B, np.complex128))


def domain_matrices(w, dec, dense=False):
    """Step 1: {subdomain: (multiplier ids, K_D)} and the LU objects."""
    out, lus = {}, {}
    for sd in dec.subs:
        D = decomp.D_matrix(dec, sd).tocsc()
        cols = np.flatnonzero(np.diff(D.indptr))
        Dc = D[:, cols].toarray()
        if dense:
            KD = Dc.T @ (np.linalg.inv(sd.A.toarray()) @ Dc)
        else:
            lu = spla.splu(sd.A.tocsc())
            lus[sd.index] = lu
            KD = domain_matrix(sd.A, Dc, lu=lu)
        out[sd.index] = (cols, KD)
    return out, lus


def assemble_K(dec, kd):
    """Step 2 (dense storage of the block-sparse K)."""
    n = len(dec.lm_edge)
    K = np.zeros((n, n), np.complex128)
    for s, (cols, KD) in kd.items():
        K[np.ix_(cols, cols)] += KD
    return K


def block_symbolic(dec):
    """Step 4: block fill of K by the elimination game on the clique graph
    (blocks adjacent when they share a subdomain), in block order."""
    nb = len(dec.blocks)
    adj = [set() for _ in range(nb)]
    for i, (a, b) in enumerate(dec.blocks):
        for j, (c, d) in enumerate(dec.blocks):
            if i != j and {a, b} & {c, d}:
                adj[i].add(j)
    pattern = set((i, i) for i in range(nb))
    parent = -np.ones(nb, np.int64)
    for j in range(nb):
        later = sorted(x for x in adj[j] if x > j)
        for i in later:
            pattern.add((i, j))
            adj[i] |= set(later) - {i}
        if later:
            parent[j] = later[0]
    return pattern, parent


def block_ldlt(K, blocks, pattern):
    """Step 5, Algorithm 1 on dense storage, touching only pattern blocks."""
    K = K.copy()
    nb = len(blocks)
    fac = {}
    for j in range(nb):
        bj = blocks[j]
        perm, Ljj, dbl, _, _ = bk.ldlt_restricted(K[np.ix_(bj, bj)])
        Djj = bk.d_matrix(dbl, len(bj))
        Lj = {}
        Xj = {}
        for i in range(j + 1, nb):
            if (i, j) not in pattern:
                continue
            Kij = K[np.ix_(blocks[i], bj)][:, perm]
            Xij = np.linalg.solve(Ljj, Kij.T).T          # K_ij P^T L_jj^{-T}
            Xj[i] = Xij
            Lj[i] = np.linalg.solve(Djj.T, Xij.T).T      # X_ij D_jj^{-1}
        for i in Lj:
            for k in Lj:
                if k <= i:
                    K[np.ix_(blocks[i], blocks[k])] -= Lj[i] @ Xj[k].T
                    if k != i:
                        K[np.ix_(blocks[k], blocks[i])] = K[np.ix_(blocks[i], blocks[k])].T
        fac[j] = (perm, Ljj, dbl, Lj)
    return fac


def block_solve(fac, blocks, g):
    """Step 6: lambda = P^T L^{-T} D^{-1} L^{-1} P g, blockwise."""
    nb = len(blocks)
    y = np.array(g, dtype=np.complex128)
    for j in range(nb):
        perm, Ljj, dbl, Lj = fac[j]
        bj = blocks[j]
        yj = y[bj][perm]
        yj = np.linalg.solve(Ljj, yj)
        y[bj] = 0
        y[bj[perm]] = yj                     # store in pivot order at permuted slots
        for i, Lij in Lj.items():
            y[blocks[i]] -= Lij @ yj
    # y[bj[perm]] now holds L^{-1}P g in pivot order; apply D^{-1} and back-solve
    x = np.zeros_like(y)
    for j in range(nb - 1, -1, -1):
        perm, Ljj, dbl, Lj = fac[j]
        bj = blocks[j]
        zj = y[bj[perm]]
        D = bk.d_matrix(dbl, len(bj))
        zj = np.linalg.solve(D, zj)
        for i, Lij in Lj.items():
            zj = zj - Lij.T @ x[blocks[i]]
        xj = np.linalg.solve(Ljj.T, zj)
        x[bj[perm]] = xj
    return x


def solve(w, f=None, dense_inverse=False, return_all=False):
    """Full D^3M solve of the workload; x (n_edges, nrhs)."""
    f = fem.rhs_planewave(w) if f is None else f
    dec = decomp.decompose(w)
    kd, lus = domain_matrices(w, dec, dense=dense_inverse)
    K = assemble_K(dec, kd)
    blocks = dec.block_lms
    pattern, _ = block_symbolic(dec)
    fac = block_ldlt(K, blocks, pattern)
    n_lm = len(dec.lm_edge)
    g = np.zeros((n_lm, f.shape[1]), np.complex128)
    ys = {}
    for sd in dec.subs:
        fi = decomp.split_rhs(dec, sd, f)
        yi = lus[sd.index].solve(fi) if lus else np.linalg.solve(sd.A.toarray(), fi)
        ys[sd.index] = (fi, yi)
        g += decomp.D_matrix(dec, sd).T @ yi
    lam = block_solve(fac, blocks, g)
    x = np.zeros((dec.grid.n_edges, f.shape[1]), np.complex128)
    copies = {}
    for sd in dec.subs:
        fi, _ = ys[sd.index]
        rhs = fi - decomp.D_matrix(dec, sd) @ lam
        Ei = lus[sd.index].solve(rhs) if lus else np.linalg.solve(sd.A.toarray(), rhs)
        for loc, e in enumerate(sd.edges):
            if dec.copies[int(e)][0] == sd.index:
                x[e] = Ei[loc]
            copies.setdefault(int(e), []).append(Ei[loc])
    mismatch = max((np.abs(np.array(v) - v[0]).max() for v in copies.values() if len(v) > 1),
                   default=0.0)
    if return_all:
        return dict(x=x, lam=lam, K=K, g=g, dec=dec, kd=kd, fac=fac, copy_mismatch=mismatch)
    return x


def solve_primal_schur(w, f=None):
    """Primal substructuring of the decomposed operators: per subdomain i with
    interior dofs I (edges held by no other subdomain) and interface dofs G,
    S = sum_i R_i^T (A_GG - A_GI A_II^{-1} A_IG) R_i and
    g = sum_i R_i^T (f_G - A_GI A_II^{-1} f_I) over the global interface
    edges (R_i: restriction to subdomain i's copies; RHS by the owner rule),
    then u_G = S^{-1} g and u_I = A_II^{-1} (f_I - A_IG u_G).  Dense Schur
    complements, for small meshes."""
    f = fem.rhs_planewave(w) if f is None else f
    dec = decomp.decompose(w)
    gam = np.array(sorted(e for e, cs in dec.copies.items() if len(cs) > 1), np.int64)
    gpos = {int(e): i for i, e in enumerate(gam)}
    nrhs = f.shape[1]
    S = np.zeros((len(gam), len(gam)), np.complex128)
    g = np.zeros((len(gam), nrhs), np.complex128)
    parts = []
    for sd in dec.subs:
        A = sd.A.toarray()
        isg = np.array([len(dec.copies[int(e)]) > 1 for e in sd.edges])
        I, G = np.flatnonzero(~isg), np.flatnonzero(isg)
        fi = decomp.split_rhs(dec, sd, f)
        AII, AIG, AGI, AGG = A[np.ix_(I, I)], A[np.ix_(I, G)], A[np.ix_(G, I)], A[np.ix_(G, G)]
        X = np.linalg.solve(AII, np.concatenate([AIG, fi[I]], axis=1)) if len(I) else np.zeros((0, len(G) + nrhs))
        rg = np.array([gpos[int(e)] for e in sd.edges[G]], np.int64)
        S[np.ix_(rg, rg)] += AGG - AGI @ X[:, :len(G)]
        g[rg] += fi[G] - AGI @ X[:, len(G):]
        parts.append((sd, I, G, rg, AII, AIG, fi))
    uG = np.linalg.solve(S, g)
    x = np.zeros((dec.grid.n_edges, nrhs), np.complex128)
    x[gam] = uG
    for sd, I, G, rg, AII, AIG, fi in parts:
        if len(I):
            x[sd.edges[I]] = np.linalg.solve(AII, fi[I] - AIG @ uG[rg])
    return x
