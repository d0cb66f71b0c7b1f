"""The dataflow POTRF's task list (emu_potrf_task_list, host only) replayed on
the CPU under the wait rules of the kernel's tasks: with any number of worker
CTAs resident, down to one, every task can eventually run, and the blocks the
tasks and the chain write form the Cholesky factor of the tile.

The kernel's CTAs fetch tasks in list order through an atomic counter; a task
holds its CTA until its inputs are published (state[r][c] counts the
operations completed on 16x16 block (r, c); a block's final count is c+1).
Here a window of W fetched tasks stands for W resident workers: at each point
one ready task of the window runs (chosen at random), then the next task of
the list is fetched.  If no fetched task is ready and the chain cannot move,
the list would stall on the GPU with W workers (the kernel's waits would time
out)."""
import numpy as np
import pytest

import paper_2408_04440_gb300 as E

PB = 16
T_LT, T_TRSM, T_UPD, T_MASTER = 0, 1, 2, 3


class Tile:
    def __init__(self, nb, seed):
        rng = np.random.default_rng(seed)
        G = rng.standard_normal((nb, nb))
        self.A = G @ G.T / nb + np.eye(nb)
        self.D = self.A.copy()
        self.nbb = nb // PB
        self.st = np.zeros((self.nbb, self.nbb), dtype=int)

    def blk(self, r, c):
        return self.D[r * PB:(r + 1) * PB, c * PB:(c + 1) * PB]

    def put(self, r, c, v):
        self.D[r * PB:(r + 1) * PB, c * PB:(c + 1) * PB] = v


def _solve_lt(L, V):
    """V L^{-T}: the solve of a sub-diagonal block against the factor L."""
    return np.linalg.solve(L, V.T).T


def task_ready(T, tk):
    k, r, c, s = (int(x) for x in tk)
    st = T.st
    if k == T_TRSM:
        # inputs of the fused panel s-1 update, then L_ss
        return ((s == 0 or (st[r, s - 1] >= s and st[s, s - 1] >= s)) and st[r, s] >= s - 1
                and st[s, s] >= s + 1)
    if k == T_UPD:
        return st[r, s] >= s + 1 and st[c, s] >= s + 1 and st[r, c] >= s
    if k == T_LT:  # batch form: step s of the chain
        return ((s < 2 or st[s, s - 2] >= s - 1) and (s < 1 or st[s, s - 1] >= s - 2) and st[s, s] >= s - 1
                and (s < 2 or st[s - 1, s - 2] >= s - 1) and (s < 1 or st[s - 1, s - 1] >= s))
    raise AssertionError(f"unexpected task kind {k}")


def task_run(T, tk):
    k, r, c, s = (int(x) for x in tk)
    if k == T_TRSM:
        v = T.blk(r, s).copy()
        if s >= 1:
            v -= T.blk(r, s - 1) @ T.blk(s, s - 1).T
        T.put(r, s, _solve_lt(T.blk(s, s), v))
        T.st[r, s] = s + 1
    elif k == T_UPD:
        T.put(r, c, T.blk(r, c) - T.blk(r, s) @ T.blk(c, s).T)
        T.st[r, c] = s + 1
    else:  # LT(s): block (s, s-1) after panel s-2, solved; block (s, s) updated and factored
        C = T.blk(s, s).copy()
        if s >= 1:
            v = T.blk(s, s - 1).copy()
            if s >= 2:
                v -= T.blk(s, s - 2) @ T.blk(s - 1, s - 2).T
            X = _solve_lt(T.blk(s - 1, s - 1), v)
            T.put(s, s - 1, X)
            T.st[s, s - 1] = s
            C -= X @ X.T
        T.put(s, s, np.linalg.cholesky(C))
        T.st[s, s] = s + 1


class Master:
    """The single-tile chain CTA: step s releases L_{s-1,s-1}, solves block
    (s, s-1) (panel s-2 applied in step s-1), publishes X_{s,s-1}, updates and
    factors block (s, s); then it waits for X_{s+1,s-1}, block (s+1, s) after
    the panels < s-1 and block (s+1, s+1) after the panels < s, and applies
    panel s-1 to block (s+1, s)."""

    def __init__(self, T):
        self.T, self.s, self.phase = T, 0, 0
        self.B = self.C = None

    def done(self):
        return self.s >= self.T.nbb

    def step(self):
        T, s = self.T, self.s
        if self.phase == 0:
            C = T.blk(0, 0).copy() if s == 0 else self.C
            if s >= 1:
                T.st[s - 1, s - 1] = s  # release L_{s-1,s-1}
                X = _solve_lt(T.blk(s - 1, s - 1), self.B)
                T.put(s, s - 1, X)
                T.st[s, s - 1] = s
                C = C - X @ X.T
            T.put(s, s, np.linalg.cholesky(C))
            self.phase = 1
            return True
        n1 = s + 1
        if n1 >= T.nbb:
            T.st[s, s] = s + 1
            self.s += 1
            return True
        st = T.st
        if (s < 1 or st[n1, s - 1] >= s) and st[n1, s] >= s - 1 and st[n1, n1] >= s:
            B = T.blk(n1, s).copy()
            if s >= 1:
                B -= T.blk(n1, s - 1) @ T.blk(s, s - 1).T
            self.B, self.C = B, T.blk(n1, n1).copy()
            self.s += 1
            self.phase = 0
            return True
        return False


class ClusterMaster:
    """The chain on a cluster of three CTAs.  Master: step s factors block
    (s, s) from C_s (formed by the first helper's step s-1) and releases
    L_{s,s}.  First helper, step s: once L_{s,s} is released, block (s+1, s)
    carries the panels < s-1, X_{s+1,s-1} is published and block (s+1, s+1)
    carries the panels < s (the last one applied by the second helper), it
    applies panel s-1 to block (s+1, s), solves and publishes X_{s+1,s} and
    forms C_{s+1} = block (s+1, s+1) minus X_{s+1,s} X_{s+1,s}^T.  Second
    helper, step s: once L_{s,s} is released, block (s+2, s) carries the
    panels < s-1 and X_{s+2,s-1} (a TRSM task) and X_{s,s-1} are published,
    it applies panel s-1, solves and publishes X_{s+2,s}; then, once block
    (s+2, s+2) carries the panels < s, it applies panel s to it.  The three
    advance independently, each on its own data."""

    def __init__(self, T):
        self.T = T
        self.s = self.sa = self.sb = 0
        self.xb = None  # the second helper's X of its current step, once solved
        self.C = {0: T.blk(0, 0).copy()}

    def done(self):
        nbb = self.T.nbb
        return self.s >= nbb and self.sa >= nbb - 1 and self.sb >= max(nbb - 2, 0)

    def step(self):
        T, st, nbb = self.T, self.T.st, self.T.nbb
        moved = False
        s = self.s
        if s < nbb and s in self.C:
            T.put(s, s, np.linalg.cholesky(self.C.pop(s)))
            st[s, s] = s + 1
            self.s += 1
            moved = True
        s, n1 = self.sa, self.sa + 1
        if n1 < nbb and st[s, s] >= s + 1 and st[n1, s] >= s - 1 and st[n1, n1] >= s and \
                (s < 1 or st[n1, s - 1] >= s):
            B = T.blk(n1, s).copy()
            if s >= 1:
                B -= T.blk(n1, s - 1) @ T.blk(s, s - 1).T
            X = _solve_lt(T.blk(s, s), B)
            T.put(n1, s, X)
            st[n1, s] = s + 1
            self.C[n1] = T.blk(n1, n1) - X @ X.T
            self.sa += 1
            moved = True
        s, n2 = self.sb, self.sb + 2
        if n2 < nbb and self.xb is None and st[s, s] >= s + 1 and st[n2, s] >= s - 1 and \
                (s < 1 or (st[n2, s - 1] >= s and st[s, s - 1] >= s)):
            B = T.blk(n2, s).copy()
            if s >= 1:
                B -= T.blk(n2, s - 1) @ T.blk(s, s - 1).T
            self.xb = _solve_lt(T.blk(s, s), B)
            T.put(n2, s, self.xb)
            st[n2, s] = s + 1
            moved = True
        if self.xb is not None and st[n2, n2] >= s:
            T.put(n2, n2, T.blk(n2, n2) - self.xb @ self.xb.T)
            st[n2, n2] = s + 1
            self.xb = None
            self.sb += 1
            moved = True
        return moved


def replay(nb, single_tile, window, seed):
    tasks = E.emu_potrf_task_list(nb, single_tile)
    T = Tile(nb, seed)
    rng = np.random.default_rng(seed + 100)
    master = None
    if single_tile:
        assert tuple(tasks[0]) == (T_MASTER, 0, 0, 0)
        assert not np.any(tasks[1:, 0] == T_MASTER)
        master = Master(T) if single_tile == 1 else ClusterMaster(T)
        tasks = tasks[1:]
    nxt, fetched = 0, []
    while nxt < len(tasks) or fetched or (master is not None and not master.done()):
        while len(fetched) < window and nxt < len(tasks):
            fetched.append(nxt)
            nxt += 1
        moved = master is not None and not master.done() and master.step()
        ready = [i for i in fetched if task_ready(T, tasks[i])]
        if ready:
            i = ready[int(rng.integers(len(ready)))]
            task_run(T, tasks[i])
            fetched.remove(i)
            moved = True
        assert moved, f"stalls with {window} workers: fetched {[tuple(tasks[i]) for i in fetched][:4]}"
    return np.abs(np.tril(T.D) - np.linalg.cholesky(T.A)).max()


@pytest.mark.parametrize("single_tile", [1, 2, 0])
@pytest.mark.parametrize("nb", [16, 32, 48, 128, 512])
def test_task_list_never_stalls_and_factors(nb, single_tile):
    for window in (1, 2, 5, 64):
        if nb == 512 and window in (2, 5):
            continue
        err = replay(nb, single_tile, window, seed=nb + window)
        assert err < 1e-10, (nb, single_tile, window, err)


def test_task_list_covers_every_update_once():
    nb = 256
    nbb = nb // PB
    for single_tile in (1, 2, 0):
        t = E.emu_potrf_task_list(nb, single_tile)
        upd = {(int(r), int(c), int(s)) for k, r, c, s in t if k == T_UPD}
        assert len(upd) == sum(1 for k in t[:, 0] if k == T_UPD)
        # every panel s updates every block (r, c), c >= s+1, except those
        # the chain (or the fused TRSM / LT update) applies: (s+1, s+1),
        # (r, s+1) for r >= s+2 (fused into TRSM(r, s+1) / LT(s+2)), and in
        # the cluster form also (s+2, s+2)
        want = {(r, c, s) for s in range(nbb) for c in range(s + 2, nbb) for r in range(c, nbb)
                if single_tile != 2 or (r, c) != (s + 2, s + 2)}
        assert upd == want
        # blocks (c+1, c) are the chain's; in the cluster form (c+2, c) too
        trsm = {(int(r), int(c)) for k, r, c, s in t if k == T_TRSM}
        assert trsm == {(r, c) for c in range(nbb) for r in range(c + (3 if single_tile == 2 else 2), nbb)}


def test_task_list_rejects_bad_sizes():
    for nb in (0, -16, 40, 4096):
        with pytest.raises(E.EmuError):
            E.emu_potrf_task_list(nb)
