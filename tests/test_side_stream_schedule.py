"""Race check of the Ozaki factorisation's two-stream schedule (host model,
no GPU).

With the Ozaki update, zgetrf forms L11^-1 of each block with its
sub-panels: per sub-panel R_s = rows/columns [s0, send) of the block
[j0, jend), L_ss^-1 comes out of the main stream's block solve of the U rows,
and two Ozaki products on a second stream give the rest of the row block,
  T = L11[R_s, j0..s0) W[..s0, ..s0),   W[R_s, j0..s0) = -L_ss^-1 T,
forked from the main stream after the sub-panel's swaps (T) and after its
block solve (the second product), joined before the next sub-panel's panel
and before U12 = W A12 (csrc/lu_host.cuh, getrf).

The model lists, in issue order, every launch of that loop with its stream
and the rectangles of memory it reads and writes (the matrix A, W, T, the
two Ozaki workspaces, ipiv).  Happens-before is program order on each stream
plus the fork edges (main -> side) and join edges (side -> main); two
launches on different streams that no chain of these orders must not touch
overlapping memory unless both only read it.  The check runs over block
widths, sub-panel widths and orders with ragged last blocks and sub-panels;
mistakes planted in the model (no join before U12, the first product forked
before the swaps, the second product without its fork after the block
solve) are caught, and the join before each panel, which is there for
speed, is shown not to be needed for correctness.
"""
import itertools

import pytest


class Op:
    def __init__(self, name, stream, reads, writes, vc):
        self.name, self.stream, self.reads, self.writes, self.vc = name, stream, reads, writes, vc


def overlap(a, b):
    """Rectangles (array, r0, r1, c0, c1), half-open."""
    return (a[0] == b[0] and a[1] < b[2] and b[1] < a[2] and a[3] < b[4] and b[3] < a[4]
            and a[1] < a[2] and a[3] < a[4] and b[1] < b[2] and b[3] < b[4])


class Schedule:
    def __init__(self):
        self.ops = {"main": [], "side": []}
        self.side_knows_main = 0  # main ops before the last fork
        self.main_knows_side = 0  # side ops before the last join

    def launch(self, stream, name, reads=(), writes=()):
        n_main, n_side = len(self.ops["main"]), len(self.ops["side"])
        if stream == "main":
            vc = {"main": n_main, "side": self.main_knows_side}
        else:
            vc = {"main": self.side_knows_main, "side": n_side}
        self.ops[stream].append(Op(name, stream, list(reads), list(writes), vc))

    def fork(self):
        self.side_knows_main = len(self.ops["main"])

    def join(self):
        self.main_knows_side = len(self.ops["side"])

    def races(self):
        out = []
        for i, a in enumerate(self.ops["main"]):
            for j, b in enumerate(self.ops["side"]):
                if b.vc["main"] > i or a.vc["side"] > j:
                    continue  # ordered
                for x, y in itertools.chain(itertools.product(a.writes, b.reads + b.writes),
                                            itertools.product(a.reads, b.writes)):
                    if overlap(x, y):
                        out.append((a.name, b.name, x, y))
        return out


def getrf_schedule(n, nb, sbw, plant=None):
    """The launches of the Ozaki getrf loop for order n, block width nb and
    sub-panel width sbw, with their memory (W and T indexed by block-local
    rows and columns)."""
    S = Schedule()
    A = lambda r0, r1, c0, c1: ("A", r0, r1, c0, c1)   # noqa: E731
    W = lambda r0, r1, c0, c1: ("W", r0, r1, c0, c1)   # noqa: E731
    T = ("T", 0, sbw, 0, nb)
    WSM, WSS = ("wsm", 0, 1, 0, 1), ("wss", 0, 1, 0, 1)
    IP = lambda k0, k1: ("ipiv", 0, 1, k0, k1)          # noqa: E731
    side_w = n > nb
    for j0 in range(0, n, nb):
        jend = min(j0 + nb, n)
        jb = jend - j0
        mkw = jend < n
        if mkw:
            S.launch("main", "identity", writes=[W(0, jb, 0, jb)])
        for s0 in range(j0, jend, sbw):
            send = min(s0 + sbw, jend)
            sb, wc = send - s0, s0 - j0
            if mkw and wc > 0 and plant != "no_panel_join":
                S.join()
            S.launch("main", f"panel {s0}", reads=[A(s0, n, s0, send)],
                     writes=[A(s0, n, s0, send), IP(s0, send)])
            t_product = ("side", f"T {s0}", [A(s0, send, j0, s0), W(0, wc, 0, wc)], [T, WSS])
            if mkw and wc > 0 and plant == "t_before_swaps":
                S.fork()
                S.launch(*t_product[:2], reads=t_product[2], writes=t_product[3])
            # the sub-panel's swaps on the block's other columns: rows s0 .. n
            S.launch("main", f"laswp {s0}", reads=[IP(s0, send), A(s0, n, j0, s0), A(s0, n, send, jend)],
                     writes=[A(s0, n, j0, s0), A(s0, n, send, jend)])
            if mkw and wc > 0 and plant != "t_before_swaps":
                S.fork()
                S.launch(*t_product[:2], reads=t_product[2], writes=t_product[3])
            # block solve: U rows right of R_s, and W[R_s, R_s] = L_ss^-1
            rw = [A(s0, send, send, jend)] + ([W(wc, wc + sb, wc, wc + sb)] if mkw else [])
            S.launch("main", f"lsolve {s0}", reads=[A(s0, send, s0, send)] + rw, writes=rw)
            if mkw and wc > 0:
                if plant != "no_second_fork":
                    S.fork()
                S.launch("side", f"W rows {s0}", reads=[W(wc, wc + sb, wc, wc + sb), T, W(wc, wc + sb, 0, wc)],
                         writes=[W(wc, wc + sb, 0, wc), WSS])
            if send < jend:
                S.launch("main", f"update {s0}",
                         reads=[A(send, n, s0, send), A(s0, send, send, jend), A(send, n, send, jend)],
                         writes=[A(send, n, send, jend), WSM])
        # the block's swaps on the columns left and right of it
        S.launch("main", f"laswp block {j0}", reads=[IP(j0, jend), A(j0, n, 0, j0), A(j0, n, jend, n)],
                 writes=[A(j0, n, 0, j0), A(j0, n, jend, n)])
        if mkw:
            if plant != "no_u12_join":
                S.join()
            S.launch("main", f"U12 {j0}", reads=[W(0, jb, 0, jb), A(j0, jend, jend, n)],
                     writes=[A(j0, jend, jend, n), WSM])
            S.launch("main", f"A22 {j0}", reads=[A(jend, n, j0, jend), A(j0, jend, jend, n), A(jend, n, jend, n)],
                     writes=[A(jend, n, jend, n), WSM])
    if side_w:
        S.join()  # the destructor's join before the workspace is freed
    return S


CASES = [(n, nb, sbw) for n in (1, 31, 96, 128, 200, 256, 300, 515) for nb in (8, 32, 48, 64, 128, 256)
         for sbw in (1, 7, 16, 24, 32) if sbw <= nb]


@pytest.mark.parametrize("n,nb,sbw", CASES)
def test_schedule_has_no_race(n, nb, sbw):
    races = getrf_schedule(n, nb, sbw).races()
    assert not races, races[:3]


@pytest.mark.parametrize("plant", ["no_u12_join", "t_before_swaps", "no_second_fork"])
def test_planted_mistakes_are_found(plant):
    found = [getrf_schedule(n, nb, sbw, plant).races() for n, nb, sbw in [(300, 128, 32), (256, 64, 16)]]
    assert all(found), plant


def test_panel_join_is_not_needed_for_correctness():
    # the join before each sub-panel's panel keeps the side stream's CTAs off
    # the SMs the cooperative panel waits for; without it the schedule is
    # still race-free (the panel and swaps touch rows below the side's R_s)
    for n, nb, sbw in [(300, 128, 32), (515, 64, 16), (256, 256, 7)]:
        assert not getrf_schedule(n, nb, sbw, "no_panel_join").races()


def test_fork_orders_side_after_main():
    # the side stream's first launch after a fork sees every main launch before it
    S = Schedule()
    S.launch("main", "a", writes=[("A", 0, 4, 0, 4)])
    S.fork()
    S.launch("side", "b", reads=[("A", 0, 4, 0, 4)])
    S.launch("main", "c", writes=[("A", 0, 4, 0, 4)])  # after the fork: concurrent with b
    assert [(r[0], r[1]) for r in S.races()] == [("c", "b")]
