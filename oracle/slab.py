"""The Crank-Nicolson step distributed over processes that each own one block
(the paper's MPI implementation, Sec. "MPI Implementation", with the exchange of
Sec. "Communication and masking of the JD and JU stages").

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the plain, serial
definition of what a multi-process N-shaped CN step computes, against which the
host-side exchange logic is checked on CPU ranks.

Layout.  G ranks, joint lines J_0 = 0 < J_1 < ... < J_G = n - 1; rank r owns the
interior rows J_r + 1 .. J_{r+1} - 1 of block r.  Every rank also holds all
joint-line values psi_J: the reduced system is solved redundantly on every rank
after one all-gather, instead of on a root process that would then send the
two support values back (one collective per step instead of two; the same
values travel).

One step, for rank r:
  1. explicit half-step d = T^dagger psi on the interior rows (their stencil
     reaches psi_{J_r} and psi_{J_r+1}, which every rank holds);
  2. Table 1 stages RD, RU, JU, JD on the local system of rows J_r .. J_{r+1},
     whose two joint rows carry only this block's share of the joint equations:
     row J_r keeps its upper coupling c and the explicit term with psi_{J_r + 1},
     row J_{r+1} its lower coupling b and the explicit term with psi_{J_{r+1} - 1};
     their diagonals start at 0.  (The two blocks' shares of a joint row add up
     to the original row, so no halo is exchanged.)
  3. all-gather of six values per rank: (c, a, d) of row J_r and (b, a, d) of row
     J_{r+1} after JU and JD -- the "values obtained on the joint lines" of the
     communication section (6 G complex numbers per step);
  4. every rank assembles the reduced system on the joint lines, adding the
     joint rows' own diagonal terms, and solves it (RS, here by Thomas);
  5. SS on the interior rows with the two support values psi_{J_r}, psi_{J_{r+1}}.

The collective is passed in: ``allgather(v)`` takes this rank's six complex
values and returns the (G, 6) array of all ranks' values in rank order.
"""
from __future__ import annotations

import numpy as np

from . import Problem, cn_matrix, default_joints, nshape_reduce, nshape_substitute, thomas, tridiag_apply

N_EXCHANGED = 6  # complex values each rank contributes per step


class SlabRank:
    """Rank r of G: its block, coefficients of T and T^dagger on its rows and the joint rows."""

    def __init__(self, prob: Problem, G: int, r: int, J=None):
        self.prob, self.G, self.r = prob, int(G), int(r)
        self.J = default_joints(prob.n, G) if J is None else np.asarray(J, dtype=np.int64)
        self.lo, self.hi = int(self.J[r]), int(self.J[r + 1])

    def interior(self, psi_full: np.ndarray) -> np.ndarray:
        return np.array(psi_full[self.lo + 1:self.hi], dtype=np.complex128)

    def step(self, psi_int: np.ndarray, psi_J: np.ndarray, E: float, allgather):
        """One CN step; returns the new (interior rows, all joint values)."""
        lo, hi, J = self.lo, self.hi, self.J
        # Coefficients for time t + dt/2 (field E); computed on the whole grid for
        # simplicity, only rows lo..hi and the joint rows are used.
        bT, aT, cT = cn_matrix(self.prob, E, +1)
        bS, aS, cS = cn_matrix(self.prob, E, -1)
        # local psi on rows lo..hi: joint values at both ends
        x = np.concatenate(([psi_J[self.r]], psi_int, [psi_J[self.r + 1]]))
        L = hi - lo + 1
        # 1. explicit half-step on the interior rows (local rows 1..L-2)
        d = tridiag_apply(bS[lo:hi + 1], aS[lo:hi + 1], cS[lo:hi + 1], x)
        # 2. the block's local system; joint rows carry this block's share only
        b = np.array(bT[lo:hi + 1])
        a = np.array(aT[lo:hi + 1])
        c = np.array(cT[lo:hi + 1])
        b[0] = 0.0
        a[0] = 0.0
        d[0] = cS[lo] * x[1]
        c[L - 1] = 0.0
        a[L - 1] = 0.0
        d[L - 1] = bS[hi] * x[L - 2]
        bw, aw, cw, dw = nshape_reduce(b, a, c, d, np.array([0, L - 1], dtype=np.int64))
        # 3. exchange
        mine = np.array([cw[0], aw[0], dw[0], bw[L - 1], aw[L - 1], dw[L - 1]], dtype=np.complex128)
        allv = np.asarray(allgather(mine), dtype=np.complex128).reshape(self.G, N_EXCHANGED)
        # 4. reduced system on the joint lines w = 0..G: the joint row's own diagonal
        # term plus the share of the block above (its JD row) and below (its JU row)
        G = self.G
        Br = np.zeros(G + 1, np.complex128)
        Ar = np.array(aT[J], dtype=np.complex128)
        Cr = np.zeros(G + 1, np.complex128)
        Dr = np.array(aS[J] * psi_J, dtype=np.complex128)
        for w in range(G + 1):
            if w > 0:  # block w-1 ends on joint w
                Br[w] = allv[w - 1, 3]
                Ar[w] += allv[w - 1, 4]
                Dr[w] += allv[w - 1, 5]
            if w < G:  # block w starts on joint w
                Cr[w] = allv[w, 0]
                Ar[w] += allv[w, 1]
                Dr[w] += allv[w, 2]
        psi_J_new = thomas(Br, Ar, Cr, Dr)
        # 5. SS on the interior rows with the support values
        xs = nshape_substitute(bw, aw, cw, dw, np.array([0, L - 1], dtype=np.int64),
                               psi_J_new[[self.r, self.r + 1]])
        return xs[1:L - 1], psi_J_new


def slab_run(prob: Problem, psi0, nsteps: int, G: int, r: int, allgather, E_mid=None, J=None):
    """nsteps distributed CN steps from psi0 (full grid, every rank reads its part);
    returns this rank's interior rows and all joint values after the last step."""
    rank = SlabRank(prob, G, r, J)
    psi0 = np.asarray(psi0, dtype=np.complex128)
    psi_int = rank.interior(psi0)
    psi_J = np.array(psi0[rank.J], dtype=np.complex128)
    for k in range(nsteps):
        E = 0.0 if E_mid is None else float(E_mid[k])
        psi_int, psi_J = rank.step(psi_int, psi_J, E, allgather)
    return psi_int, psi_J


def assemble(J, interiors, psi_J) -> np.ndarray:
    """Full grid from every rank's interior rows and the joint values."""
    J = np.asarray(J, dtype=np.int64)
    out = np.empty(int(J[-1]) + 1, np.complex128)
    out[J] = psi_J
    for r, v in enumerate(interiors):
        out[J[r] + 1:J[r + 1]] = v
    return out
