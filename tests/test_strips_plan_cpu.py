"""Halo bookkeeping of the strip-decomposed field, as two gloo ranks on CPU.

ofv_compute_strips splits one field into horizontal strips that would live
on separate GPUs (rank r holds strip r).  Each rank asks the library for its
own plan (ofv_strip_plan: a host-only call) and the ranks exchange what they
own and what they read, as they would before a multi-GPU run.  The checks:
the owned rows partition every level in whole tile rows; every row a rank
reads of a field outside its own rows is owned by another rank, which
therefore sends it (the two sides compute the same row sets); the rows a
strip up-samples from the coarser level are held after the coarse level's
exchange; and every strip computes the image rows its tiles read.  The
decomposition is exchanged, not assumed: each rank sees only the other's
plan through the process group.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

CASES = [  # H, W, PSL, KR, NR, prefilter, max_disp, tile_edge (0: the radius's default)
    (4096, 5120, 2, 4, 0, 0, 8, 0), (1024, 1024, 2, 4, 0, 0, 6, 0), (300, 200, 2, 4, 2, 1, 6, 0),
    (2048, 2048, 2, 10, 2, 0, 16, 0), (97, 131, 1, 3, 0, 0, 4, 0), (600, 80, 3, 2, 1, 0, 20, 0),
    (1024, 1024, 2, 4, 0, 0, 6, 32), (700, 900, 2, 6, 0, 0, 8, 32), (2048, 2048, 2, 10, 2, 0, 16, 32),
]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import paper_2509_25924_gb300 as ofv
    results = []
    for (H, W, psl, kr, nr, pf, md, te) in CASES:
        p = ofv.ofv_default_params(levels_psl=psl, kernel_radius=kr, norm_radius=nr, prefilter=pf, tile_edge=te)
        mine = [ofv.ofv_strip_plan(H, W, p, ws, md, l, rank) for l in range(psl + 1)]
        plans = [None] * ws
        dist.all_gather_object(plans, mine)  # rank k's plan, as rank k computed it
        results.append(_check(ofv, H, W, psl, kr, nr, pf, md, te, rank, ws, plans))
    dist.barrier()
    q.put((rank, results))
    dist.destroy_process_group()


def _inside(r, outer):
    return r[0] >= r[1] or (outer[0] <= r[0] and r[1] <= outer[1])


def _check(ofv, H, W, psl, kr, nr, pf, md, te, rank, ws, plans):
    ts = te or (48 if kr <= 5 else 64)  # the block kernel's tile edge
    Hs = [H]
    for _ in range(psl):
        Hs.append((Hs[-1] + 1) // 2)
    for l in range(psl + 1):
        own = [plans[k][l]["own"] for k in range(ws)]
        # a partition of the level in order, in whole tile rows
        assert own[0][0] == 0 and own[-1][1] == Hs[l]
        for k in range(ws - 1):
            assert own[k][1] == own[k + 1][0]
        for a, b in own:
            assert a % ts == 0 and (b % ts == 0 or b == Hs[l])
        me = plans[rank][l]
        if me["own"][0] < me["own"][1]:
            # the window halo of the field, clipped to the level
            assert me["fld"] == (max(0, me["own"][0] - kr), min(Hs[l], me["own"][1] + kr))
            # the rows read outside the own rows are owned by the others, who send
            # exactly fld(me) n own(them)
            recv = set(range(*me["fld"])) - set(range(*me["own"]))
            sent = set()
            for k in range(ws):
                if k != rank:
                    r = plans[k][l]["own"]
                    sent |= set(range(max(r[0], me["fld"][0]), min(r[1], me["fld"][1])))
            assert recv == sent
            # the images the tiles read: own rows +- (KR + warp reach + stencil)
            margin = kr + 4 + 2
            assert _inside((max(0, me["own"][0] - margin), min(Hs[l], me["own"][1] + margin)), me["img"])
        if l + 1 <= psl and me["fld"][0] < me["fld"][1]:
            # up-sampling to level l reads coarse rows y/2, y/2 + 1 of level l+1
            up = me["up"]
            assert up[0] <= me["fld"][0] // 2 and up[1] >= min(Hs[l + 1], (me["fld"][1] - 1) // 2 + 2)
            coarse_own = [plans[k][l + 1]["own"] for k in range(ws)]
            held = set()
            for r in coarse_own:
                held |= set(range(*r))
            assert set(range(*up)) <= held
        if l >= 1 and me["img"][0] < me["img"][1]:
            # a level-l image row i reads level l-1 rows 2i-2 .. 2i+2 (clamped)
            fine = plans[rank][l - 1]["img"]
            assert _inside((max(0, 2 * me["img"][0] - 2), min(Hs[l - 1], 2 * me["img"][1] + 1)), fine)
            assert fine[0] % 2 == 0
    # level 0 is ingested over the image rows plus the reach of NR and the pre-filter
    ing, img0 = plans[rank][0]["ingest"], plans[rank][0]["img"]
    reach = nr + (2 if pf else 0)
    assert _inside((max(0, img0[0] - reach), min(H, img0[1] + reach)), ing)
    return True


def test_two_ranks_agree_on_the_strip_halos():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _ in res] == [0, 1] and all(all(x) for _, x in res)


def test_single_strip_owns_everything_and_reads_nothing_else():
    import paper_2509_25924_gb300 as ofv
    p = ofv.ofv_default_params()
    for l in range(3):
        pl = ofv.ofv_strip_plan(1000, 700, p, 1, 8, l, 0)
        Hl = [1000, 500, 250][l]
        assert pl["own"] == (0, Hl) and pl["fld"] == (0, Hl) and pl["img"] == (0, Hl)


def test_invalid_strip_requests_are_rejected():
    import paper_2509_25924_gb300 as ofv
    p = ofv.ofv_default_params()
    for args in ((1000, 700, p, 0, 8, 0, 0), (1000, 700, p, 2, 8, 0, 2), (1000, 700, p, 2, 8, 3, 0),
                 (1000, 700, p, 2, -1, 0, 0)):
        with pytest.raises(ofv.OfvError) as ei:
            ofv.ofv_strip_plan(*args)
        assert ei.value.status == ofv.OFV_ERR_INVALID_ARG
    with pytest.raises(ofv.OfvError) as ei:
        ofv.ofv_strip_plan(1000, 700, ofv.ofv_default_params(kernel_radius=12), 2, 8, 0, 0)
    assert ei.value.status == ofv.OFV_ERR_UNSUPPORTED
