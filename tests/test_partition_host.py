"""Domain decomposition, host side (CPU, no device work): the partitioner, the parts' halo lists
and their consistency across ranks, checked on one process and with two gloo ranks that exchange
their halo lists and halo payloads.

The payload exchanged is geometric: every rank writes, for each halo interface, the physical
coordinates of its own side's flux points in the interface's slot order (the order the library
stores traces in, from the documented face-table orientation codes), and the peer must receive
exactly its own side's coordinates (up to the periodic translation): the k-th entry a rank sends
to a peer is the k-th entry the peer receives, and the slots of both sides meet point by point.
"""
import os
import socket
import sys

import numpy as np
import pytest

from oracle.hexfr import HexFR
from paper_2308_06605_gb300 import fr, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TWO_PI = 2 * np.pi


def _mesh():
    return I.hex_box_mesh((4, 3, 3), seed=5, shuffle=True, rotate=True, perturb=0.05)


def test_partition_is_balanced_deterministic_and_covers_the_mesh():
    d = _mesh()
    for n_parts in (1, 2, 3, 4, 7):
        part = fr.partition(d, 2, n_parts)
        assert np.array_equal(part, fr.partition(d, 2, n_parts))
        counts = np.bincount(part, minlength=n_parts)
        assert counts.sum() == 36 and counts.min() >= 1
        assert counts.max() - counts.min() <= 1 + 36 // n_parts // 4, counts
        owned = np.concatenate([fr.part_inspect(d, 2, part, r)["elem_global"] for r in range(n_parts)])
        assert np.array_equal(np.sort(owned), np.arange(36))


def test_halo_lists_match_between_every_pair_of_parts():
    d = _mesh()
    n_parts = 4
    part = fr.partition(d, 2, n_parts)
    info = [fr.part_inspect(d, 2, part, r) for r in range(n_parts)]
    g = fr.inspect(d, 2)
    n_two_sided = g["n_iface"]
    seen = np.zeros(n_two_sided, dtype=int)
    for r, h in enumerate(info):
        for k, q in enumerate(h["peers"]):
            mine = h["gid"][h["peer_begin"][k]:h["peer_begin"][k + 1]]
            hq = info[q]
            kk = list(hq["peers"]).index(r)
            theirs = hq["gid"][hq["peer_begin"][kk]:hq["peer_begin"][kk + 1]]
            assert np.array_equal(mine, theirs)
            assert np.all(np.diff(mine) > 0)
            seen[mine] += 1
    # Each global interface is internal to one part or shared by exactly two.
    ef = g["ef"]
    side_elem = {}
    for e in range(ef.shape[0]):
        for f in range(6):
            side_elem.setdefault(int(ef[e, f]) >> 4, []).append(e)
    for I_ in range(n_two_sided):
        parts = {int(part[e]) for e in side_elem[I_]}
        assert seen[I_] == (0 if len(parts) == 1 else 2)
    # Two-sided interfaces of a part = internal + halo ones.
    for r, h in enumerate(info):
        internal = sum(1 for I_ in range(n_two_sided) if {int(part[e]) for e in side_elem[I_]} == {r})
        assert h["n_iface"] == internal + h["n_halo"]


def test_partition_refusals():
    d = _mesh()
    with pytest.raises(fr.FRError) as ei:
        fr.partition(d, 2, 0)
    assert ei.value.status == fr.FR_EINVAL
    with pytest.raises(fr.FRError) as ei:
        fr.partition(d, 2, 37)
    assert ei.value.status == fr.FR_EINVAL
    with pytest.raises(fr.FRError) as ei:
        fr.part_inspect(d, 2, np.full(36, -1, np.int32), 0)
    assert ei.value.status == fr.FR_EINVAL
    with pytest.raises(fr.FRError) as ei:
        fr.part_inspect(d, 2, np.zeros(36, np.int32), 1)        # part 1 owns nothing
    assert ei.value.status == fr.FR_EINVAL


@pytest.mark.parametrize("split", ["checker", "all"])
def test_halo_lists_match_on_mixed_meshes(split):
    """Hexahedra and prisms (checkerboard columns, or every column split): the parts own every
    element once (hexahedra first, then prisms, each in input order), the halo lists of every
    pair agree, and each global interface is internal to one part or shared by exactly two."""
    d = I.hex_box_mesh((4, 4, 3), prisms=split, seed=2)
    p, n_parts = 3, 3
    part = fr.partition(d, p, n_parts)
    g = fr.inspect(d, p)
    E, Ep = g["n_elem"], g["n_prism"]
    info = [fr.part_inspect(d, p, part, r) for r in range(n_parts)]
    owned = np.concatenate([h["elem_global"] for h in info])
    assert np.array_equal(np.sort(owned), np.arange(E + Ep))
    for r, h in enumerate(info):
        eg = np.asarray(h["elem_global"])
        assert np.array_equal(eg, np.sort(eg)) and np.all(part[eg] == r)
    side_elem = {}
    for e in range(E):
        for f in range(6):
            side_elem.setdefault(int(g["ef"][e, f]) >> 4, []).append(e)
    for ep in range(Ep):
        for f in range(5):
            side_elem.setdefault(int(g["ef_prism"][ep, f]) >> 4, []).append(E + ep)
    seen = np.zeros(g["n_iface"], dtype=int)
    for r, h in enumerate(info):
        for k, q in enumerate(h["peers"]):
            mine = h["gid"][h["peer_begin"][k]:h["peer_begin"][k + 1]]
            kk = list(info[q]["peers"]).index(r)
            theirs = info[q]["gid"][info[q]["peer_begin"][kk]:info[q]["peer_begin"][kk + 1]]
            assert np.array_equal(mine, theirs) and np.all(np.diff(mine) > 0)
            seen[mine] += 1
    for I_ in range(g["n_iface"]):
        assert seen[I_] == (0 if len({int(part[e]) for e in side_elem[I_]}) == 1 else 2)
    for r, h in enumerate(info):
        internal = sum(1 for I_ in range(g["n_iface"]) if {int(part[e]) for e in side_elem[I_]} == {r})
        assert h["n_iface"] == internal + h["n_halo"]


def _part_work(desc, p, part, n_parts, cost):
    g = fr.inspect(desc, p)
    E = g["n_elem"]
    w = np.r_[np.full(E, g["n_pts"] * cost[0]), np.full(g["n_prism"], g["n_pts_prism"] * cost[1])]
    return np.bincount(part, weights=w, minlength=n_parts)


def test_cost_weighted_partition_balances_work_on_mixed_meshes():
    """fr_partition_cost: unit costs reproduce fr_partition; with a prism point costing more (the
    algorithmic flops per point of each type) the parts' work is at least as balanced as with the
    point-count partition, and the cut moves."""
    from paper_2308_06605_gb300 import perfmodel as PM
    d = I.hex_box_mesh((6, 5, 4), prisms="checker", seed=7)
    p, n_parts = 4, 4
    assert np.array_equal(fr.partition(d, p, n_parts, cost=(1.0, 1.0)), fr.partition(d, p, n_parts))
    cost = PM.point_cost(p)
    assert cost[1] > 2 * cost[0]
    by_points = fr.partition(d, p, n_parts)
    by_work = fr.partition(d, p, n_parts, cost=cost)
    assert not np.array_equal(by_points, by_work)
    imb = lambda w: w.max() / w.mean()                                   # noqa: E731
    assert imb(_part_work(d, p, by_work, n_parts, cost)) <= imb(_part_work(d, p, by_points, n_parts, cost)) + 1e-12
    assert imb(_part_work(d, p, by_work, n_parts, cost)) < 1.1
    for bad in ((0.0, 1.0), (1.0, -2.0), (float("nan"), 1.0), (1.0, float("inf"))):
        with pytest.raises(fr.FRError) as ei:
            fr.partition(d, p, n_parts, cost=bad)
        assert ei.value.status == fr.FR_EINVAL


def _slot(code, a, b, N):
    if code & 4:
        a, b = b, a
    if code & 1:
        a = N - 1 - a
    if code & 2:
        b = N - 1 - b
    return a + N * b


def halo_payload(d, p, part, rank):
    """[n_halo][Nf][3]: this rank's side's flux-point coordinates of each halo interface, in the
    interface's slot order, in halo-list order."""
    h = fr.part_inspect(d, p, part, rank)
    ef = fr.inspect(d, p)["ef"]
    xf = HexFR(d, I.tgv_physics(), p).xf          # [E][6][Nf][3], face point a + N b
    N = p + 1
    where = {}
    for e in range(ef.shape[0]):
        if part[e] != rank:
            continue
        for f in range(6):
            where[int(ef[e, f]) >> 4] = (e, f, int(ef[e, f]) & 7)
    out = np.zeros((h["n_halo"], N * N, 3))
    for k, gid in enumerate(h["gid"]):
        e, f, code = where[int(gid)]
        for b in range(N):
            for a in range(N):
                out[k, _slot(code, a, b, N)] = xf[e, f, a + N * b]
    return h, out


def _check_received(mine, got):
    dlt = got - mine
    dlt -= TWO_PI * np.round(dlt / TWO_PI)         # periodic interfaces meet across the box
    return np.abs(dlt).max()


def test_single_process_payload_exchange_meets_point_by_point():
    d = _mesh()
    p, n_parts = 2, 3
    part = fr.partition(d, p, n_parts)
    data = [halo_payload(d, p, part, r) for r in range(n_parts)]
    for r, (h, mine) in enumerate(data):
        for k, q in enumerate(h["peers"]):
            hq, theirs = data[q]
            kk = list(hq["peers"]).index(r)
            got = theirs[hq["peer_begin"][kk]:hq["peer_begin"][kk + 1]]
            assert _check_received(mine[h["peer_begin"][k]:h["peer_begin"][k + 1]], got) < 1e-12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2308_06605_gb300 import fr as F, inputs as In
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        d = In.hex_box_mesh((4, 3, 3), seed=5, shuffle=True, rotate=True, perturb=0.05)
        p = 2
        part = F.partition(d, p, world)
        h, mine = halo_payload(d, p, part, rank)
        worst = 0.0
        for k, q in enumerate(h["peers"]):
            b, e = h["peer_begin"][k], h["peer_begin"][k + 1]
            # Halo lists first (the peer's list for this rank must be the same interfaces) ...
            gid = torch.from_numpy(h["gid"][b:e].copy())
            other = torch.empty_like(gid)
            reqs = [dist.isend(gid, int(q)), dist.irecv(other, int(q))]
            for rq in reqs:
                rq.wait()
            assert torch.equal(gid, other)
            # ... then the payload, as a stage exchanges traces.
            send = torch.from_numpy(np.ascontiguousarray(mine[b:e]))
            recv = torch.empty_like(send)
            reqs = [dist.isend(send, int(q)), dist.irecv(recv, int(q))]
            for rq in reqs:
                rq.wait()
            worst = max(worst, _check_received(mine[b:e], recv.numpy()))
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
            fh.write(f"{h['n_halo']} {float(worst)!r}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halo_lists_and_payloads(tmp_path):
    torch = pytest.importorskip("torch")
    world = 2
    torch.multiprocessing.spawn(_gloo_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        n_halo, worst = open(tmp_path / f"r{r}.txt").read().split()
        assert int(n_halo) > 0 and float(worst) < 1e-12


def test_payload_check_catches_ignored_orientation(monkeypatch):
    """Planted mistake: slots taken without the orientation code; the payload check must fail."""
    import test_partition_host as T
    monkeypatch.setattr(T, "_slot", lambda code, a, b, N: a + N * b)
    d = _mesh()
    p = 2
    part = fr.partition(d, p, 2)
    (h0, m0), (h1, m1) = T.halo_payload(d, p, part, 0), T.halo_payload(d, p, part, 1)
    assert _check_received(m0, m1) > 1e-3
