"""Deadlock check of the cooperative panels' named-barrier protocols (host
model, no GPU): k_panel_team (TD, QD) and k_panel_coop (DD).

The kernel's warps are modelled as threads that execute, per panel column,
the same sequence of barrier operations as csrc/panel_team.cuh and
csrc/panel_coop.cuh:
producers `bar.arrive`, consumers `bar.sync`, a phase completing when the
barrier's thread count has arrived.  Every path is covered: ordinary columns,
zero pivots (no elimination), and a timed-out exchange at the first, a middle
and the last column (the factor team releases the update team at its next go
signal), and columns whose candidate keys are near (the full-key
comparison adds barrier phases that every warp of the group takes).  A wait
that does not complete within two seconds is a deadlock.
"""
import threading

import pytest

COUNTS = {"MAIN": 128, "RCP": 64, "DONE": 224, "PUB": 96, "SWAP": 128, "GO": 256, "ALL": 256}


class NamedBarrier:
    def __init__(self, count):
        self.count, self.arrived, self.gen = count, 0, 0
        self.cv = threading.Condition()

    def _arrive(self, n):
        self.arrived += n
        if self.arrived > self.count:
            raise RuntimeError("more arrivals than the barrier's count")
        if self.arrived == self.count:
            self.arrived = 0
            self.gen += 1
            self.cv.notify_all()
            return True
        return False

    def sync(self, n=32):
        with self.cv:
            g = self.gen
            if self._arrive(n):
                return
            if not self.cv.wait_for(lambda: self.gen != g, timeout=2.0):
                raise RuntimeError("deadlock")

    def arrive(self, n=32):
        with self.cv:
            self._arrive(n)


def run_protocol(nb, zero_cols, err_col, near_cols=frozenset()):
    B = {k: NamedBarrier(v) for k, v in COUNTS.items()}
    sh = {"ok": 1, "zero": 0}
    errors, lock = [], threading.Lock()

    def update_warp(w):
        for jc in range(nb):
            B["GO"].sync()
            if not sh["ok"]:
                break
            B["DONE"].arrive()
        B["ALL"].sync()

    def factor_warp(w):
        B["GO"].arrive()
        for jc in range(nb):
            B["MAIN"].sync()  # keys: warp results (k0)
            B["MAIN"].sync()  # keys: the CTA's candidate by k0
            B["MAIN"].sync()  # keys: near flags
            if jc in near_cols:
                B["MAIN"].sync()  # full keys of the near rows: warp results
            B["MAIN"].sync()  # keys: CTA result
            if w < 3:
                if w < 2:
                    B["RCP"].sync()
                    B["RCP"].sync()
                B["DONE"].sync()
                B["PUB"].sync()
                B["SWAP"].arrive()
            else:
                B["SWAP"].sync()
                with lock:
                    if jc == err_col:
                        sh["ok"] = 0
                    sh["zero"] = 1 if jc in zero_cols else 0
            B["MAIN"].sync()
            if not sh["ok"]:
                if jc + 1 < nb:
                    B["GO"].arrive()
                break
            if sh["zero"]:
                if jc + 1 < nb:
                    B["MAIN"].sync()
                    B["GO"].arrive()
                continue
            B["MAIN"].sync()  # multiplier products
            if jc + 1 < nb:
                B["MAIN"].sync()  # multipliers final
                B["GO"].arrive()
                B["MAIN"].sync()  # next column's products
            B["MAIN"].sync()  # end of the column
        B["ALL"].sync()

    def wrap(f, w):
        try:
            f(w)
        except Exception as e:  # noqa: BLE001
            errors.append((w, repr(e)))

    ts = [threading.Thread(target=wrap, args=(factor_warp if w < 4 else update_warp, w)) for w in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return errors


@pytest.mark.parametrize("nb", [1, 2, 3, 5, 32])
def test_panel_team_protocol_deadlock_free(nb):
    cases = [((), -1), ((0,), -1), ((nb - 1,), -1), (tuple(range(nb)), -1),
             ((), 0), ((), nb - 1), ((1,), nb // 2)]
    for zero_cols, err_col in cases:
        for near in (set(), {0, nb - 1}, set(range(0, nb, 2))):
            assert run_protocol(nb, set(zero_cols), err_col, near) == [], (nb, zero_cols, err_col, near)


def test_protocol_model_detects_a_missing_arrival():
    """The model itself: dropping the factor team's first go signal deadlocks."""
    B = NamedBarrier(64)
    out = []

    def waiter():
        try:
            B.sync()
        except RuntimeError as e:
            out.append(str(e))

    t = threading.Thread(target=waiter)
    t.start()
    t.join()
    assert out == ["deadlock"]


def run_coop_protocol(nb, zero_cols, err_col, near_cols=frozenset()):
    """k_panel_coop: __syncthreads (all 8 warps), bar 1 (warps 0, 1, 4, 5:
    the reciprocal), bar 2 (warps 0, 1, 2, 7: release of the flag), bar 3
    (warps 2 and 7 arrive, warp 3 waits before its swap)."""
    B = {"ALL": NamedBarrier(256), "B1": NamedBarrier(128), "B2": NamedBarrier(128), "B3": NamedBarrier(96)}
    sh = {"ok": 1, "zero": 0}
    errors, lock = [], threading.Lock()

    def warp(w):
        B["ALL"].sync()                       # rows loaded
        for jc in range(nb):
            B["ALL"].sync(); B["ALL"].sync()  # keys: block argmax of k0
            B["ALL"].sync()                   # keys: the candidate by k0
            B["ALL"].sync()                   # keys: __syncthreads_or of the near flags
            if jc in near_cols:
                B["ALL"].sync(); B["ALL"].sync()  # full keys of the near rows: block argmax
            B["ALL"].sync()                   # keys: the CTA's candidate
            if w in (0, 1, 4, 5):
                B["B1"].sync(); B["B1"].sync()
            elif w in (2, 7):
                B["B3"].arrive()
            if w in (0, 1, 2, 7):
                B["B2"].sync()
            if w == 3:
                B["B3"].sync()
                with lock:
                    if jc == err_col:
                        sh["ok"] = 0
                    sh["zero"] = 1 if jc in zero_cols else 0
            B["ALL"].sync()                   # update and exchange done
            if not sh["ok"]:
                return
            if sh["zero"]:
                B["ALL"].sync()
                continue
            B["ALL"].sync()                   # multiplier products
            B["ALL"].sync()                   # multipliers
            if jc + 1 < nb:
                B["ALL"].sync()               # next column's products
            B["ALL"].sync()                   # end of the column

    def wrap(w):
        try:
            warp(w)
        except Exception as e:  # noqa: BLE001
            errors.append((w, repr(e)))

    ts = [threading.Thread(target=wrap, args=(w,)) for w in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return errors


@pytest.mark.parametrize("nb", [1, 2, 3, 5, 32])
def test_panel_coop_protocol_deadlock_free(nb):
    cases = [((), -1), ((0,), -1), ((nb - 1,), -1), (tuple(range(nb)), -1),
             ((), 0), ((), nb - 1), ((1,), nb // 2)]
    for zero_cols, err_col in cases:
        for near in (set(), {0, nb - 1}, set(range(0, nb, 2))):
            assert run_coop_protocol(nb, set(zero_cols), err_col, near) == [], (nb, zero_cols, err_col, near)
