"""Domain decomposition of the scheme on the oracle (CPU): sub-domains that
exchange a two-cell halo after every RK stage and combine their CFL maxima
step the whole domain bit for bit, in one process and as two or four gloo
ranks that exchange their halos as messages. The stencil of Section 3 reads two
cells along x and y per stage; eq:cfl's maximum is an exact reduction."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_1912_02457_gb300 import synth  # noqa: E402

STEPS = 8


def _workload():
    """Coastal 48 x 40: nested S, N and W edges (tide frames sampled along
    the edges), an east wall, land, varying f, drag, and gridded wind that
    varies in x, y and time (sampled at the whole domain's positions)."""
    from helpers import gridded_wind
    wl = synth.coastal(48, 40, dtype=np.float64)
    wl.wind = gridded_wind(5, 4)
    return wl


@pytest.fixture(scope="module")
def whole():
    from oracle import decomp
    return decomp.run_split(_workload(), 1, 1, STEPS)


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_the_whole_domain_step_is_the_oracle_step(whole):
    from oracle import Oracle
    (e, u, v), (t, dt) = whole
    ref = Oracle(_workload()).run(STEPS)
    # the same formulas in the same order (the oracle is compiled without
    # multiply-add contraction, numpy rounds each operation too)
    assert _same((e, u, v), ref[:3]) and (t, dt) == (ref[3], ref[4])


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2), (3, 2), (2, 3)])
def test_split_equals_whole_bit_for_bit(whole, px, py):
    from oracle import decomp
    out, clock = decomp.run_split(_workload(), px, py, STEPS)
    assert _same(out, whole[0]) and clock == whole[1]


def test_split_reaches_a_horizon_like_the_oracle():
    # the horizon falls inside the steps: the last step is shortened to end
    # on it and the later ones are no-ops, split or whole, as in orc_run
    from oracle import Oracle, decomp
    wl = _workload()
    t_end = 5.0
    ref = Oracle(wl).run(STEPS, t_end=t_end)
    assert ref[3] == t_end
    for px, py in ((1, 1), (2, 2)):
        out, (t, _) = decomp.run_split(wl, px, py, STEPS, t_end=t_end)
        assert t == t_end and _same(out, ref[:3])


def test_a_one_cell_halo_is_not_enough(whole, monkeypatch):
    # the stage reads two cells on each side: one halo cell breaks the split
    from oracle import decomp
    part = synth.partition
    monkeypatch.setattr(synth, "partition", lambda nx, ny, px, py, halo=2: part(nx, ny, px, py, 1))
    out, _ = decomp.run_split(_workload(), 2, 2, STEPS)
    assert max(np.abs(a - b).max() for a, b in zip(out, whole[0])) > 1e-3


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2)])
def test_windows_sample_the_forcing_at_whole_domain_positions(whole, monkeypatch, px, py):
    # a window that samples wind and nesting frames at its own positions
    # steps a different problem
    from oracle import Oracle, decomp
    init = decomp.SubOracle.__init__

    def own_positions(self, wl, part):
        init(self, wl, part)
        self.orc = Oracle(self.win)
    monkeypatch.setattr(decomp.SubOracle, "__init__", own_positions)
    out, _ = decomp.run_split(_workload(), px, py, STEPS)
    assert max(np.abs(a - b).max() for a, b in zip(out, whole[0])) > 1e-3


def test_partition_covers_the_domain_once():
    parts = synth.partition(37, 23, 3, 4)
    seen = np.zeros((23, 37), int)
    for p in parts:
        x0, x1, y0, y1 = p["own"]
        assert x1 - x0 >= 2 and y1 - y0 >= 2
        seen[y0:y1, x0:x1] += 1
        w = p["win"]
        assert w[0] == x0 - 2 * p["cut"][2] and w[1] == x1 + 2 * p["cut"][3]
        assert w[2] == y0 - 2 * p["cut"][0] and w[3] == y1 + 2 * p["cut"][1]
    assert (seen == 1).all()
    with pytest.raises(ValueError):
        synth.partition(5, 40, 3, 1)


def test_window_cuts_the_workload():
    wl = _workload()
    parts = synth.partition(wl.nx, wl.ny, 2, 2)
    p = parts[3]                                  # north-east block: cuts to its south and west
    w = synth.window(wl, p)
    x0, x1, y0, y1 = p["win"]
    assert (w.nx, w.ny) == (x1 - x0, y1 - y0) and w.H.shape == (w.ny + 1, w.nx + 1)
    assert np.array_equal(w.H, wl.H[y0:y1 + 1, x0:x1 + 1])
    assert np.array_equal(w.eta, wl.eta[y0:y1, x0:x1]) and np.array_equal(w.f, wl.f[y0:y1, x0:x1])
    # cut edges become walls, the whole domain's own edges keep their kind
    assert w.bc == (synth.BC_WALL, wl.bc[1], synth.BC_WALL, wl.bc[3])
    assert w.boundary is wl.boundary and w.wind is wl.wind
    per = wl.copy()
    per.bc = (synth.BC_PERIODIC,) * 4
    with pytest.raises(ValueError):
        synth.window(per, p)


# ---------------------------------------------------------------------------
# two gloo ranks, one sub-domain each

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _overlap(a, b):
    """Cells of box a (x0, x1, y0, y1) that lie in box b, or None."""
    x0, x1 = max(a[0], b[0]), min(a[1], b[1])
    y0, y1 = max(a[2], b[2]), min(a[3], b[3])
    return (x0, x1, y0, y1) if x0 < x1 and y0 < y1 else None


def _rank_main(rank, ws, port, px, py, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch
    import torch.distributed as dist
    from oracle import decomp
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    wl = _workload()
    parts = synth.partition(wl.nx, wl.ny, px, py)
    me = parts[rank]
    sub = decomp.SubOracle(wl, me)
    wx0, wy0 = me["win"][0], me["win"][2]

    def exchange(subs, which):
        # every pair of ranks swaps the cells of each one's window that the
        # other owns (the halo strips; corners too, in a 2-D split)
        fields = subs[0].fields(which)
        reqs, inbox = [], []
        for other in parts:
            if other["rank"] == rank:
                continue
            out = _overlap(other["win"], me["own"])
            if out:
                x0, x1, y0, y1 = out
                buf = torch.from_numpy(np.stack([a[y0 - wy0:y1 - wy0, x0 - wx0:x1 - wx0] for a in fields]).copy())
                reqs.append(dist.isend(buf, dst=other["rank"]))
            into = _overlap(me["win"], other["own"])
            if into:
                x0, x1, y0, y1 = into
                buf = torch.empty((3, y1 - y0, x1 - x0), dtype=torch.float64)
                reqs.append(dist.irecv(buf, src=other["rank"]))
                inbox.append((into, buf))
        for r in reqs:
            r.wait()
        for (x0, x1, y0, y1), buf in inbox:
            for a, b in zip(fields, buf.numpy()):
                a[y0 - wy0:y1 - wy0, x0 - wx0:x1 - wx0] = b

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    t, dt = decomp.step([sub], STEPS, wl.t0, wl.params.courant, exchange, reduce_max)
    r, c = sub.own_slices()
    q.put((rank, me["own"], [a[r, c].copy() for a in sub.Q], (t, dt)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2)])
def test_gloo_ranks_equal_the_whole_domain(whole, px, py):
    # two ranks split along x or y; four ranks in 2 x 2, whose window
    # corners come from the diagonal neighbour
    import torch.multiprocessing as mp
    from oracle import build
    build()                                  # compiled once, before the ranks start
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ws = px * py
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, px, py, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = [np.full_like(a, np.nan) for a in whole[0]]
    for _, (x0, x1, y0, y1), arrays, clock in got:
        assert clock == whole[1]
        for o, a in zip(out, arrays):
            o[y0:y1, x0:x1] = a
    assert _same(out, whole[0])
