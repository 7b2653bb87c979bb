"""Accuracy against the numbers the paper prints: on synthetic stand-ins of
its Rankine test images (Sec. 4.1: 1024 x 1024 px, particles of radius
1.5 px, concentration in particles per 16 x 16 px window, no noise), the
estimator with the best parameters of Table 3 must stay within the error
range Table 4 reports for those best cases (<Err> from 0.048 to 0.27 px, the
spatial mean of |V - V_true|).

The images are ours, not the third-party generator's (no out-of-plane
motion, our particle rendering and the midpoint convention of the design
notes), so the comparison is with the paper's upper bound, on the cases
with a maximum displacement of 8 and 16 px.  Measured with the oracle: all
12 such cases between 0.049 and 0.064 px; over all 24 rows of Table 3,
22 stay within the range (the two 32 px cases at R = 75 and 100 px give
0.34 and 0.27 px).
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rankine_best_configs.txt")
N = 1024


def _table():
    rows, rng = [], None
    for line in open(GOLDEN):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "err_range_px":
            rng = (float(t[1]), float(t[2]))
            continue
        R, D, piw, kr, nr, psl, it = (int(x) for x in t[:7])
        rows.append(dict(R=R, D=D, piw=piw, kr=kr, nr=nr, psl=psl, it=it, dr=float(t[7])))
    return rows, rng


ROWS, ERR_RANGE = _table()
SMALL_D = [r for r in ROWS if r["D"] <= 16]


def _pair(r):
    f = synth.rankine_field(N, N, r["R"], r["D"])
    I1, I2 = synth.particle_pair(N, N, f, ppp=r["piw"] / 256.0, dmin=3.0, dmax=3.0, seed=r["R"] + r["D"],
                                 noise=0.0, bits=12, kind=synth.OUT_U16, field_max=r["D"])
    return I1, I2, f.grid(N, N)


def test_table_transcription_is_consistent():
    """24 rows (6 radii x 4 displacements, Table 1's grid) and D/R as printed."""
    assert len(ROWS) == 24 and ERR_RANGE == (0.048, 0.27)
    assert sorted({r["R"] for r in ROWS}) == [12, 25, 50, 75, 100, 150]
    assert sorted({r["D"] for r in ROWS}) == [8, 16, 24, 32]
    for r in ROWS:
        assert abs(r["D"] / r["R"] - r["dr"]) < 0.006, r
        assert 2 <= r["kr"] <= 7 and 1 <= r["nr"] <= 4 and 2 <= r["psl"] <= 4 and 1 <= r["it"] <= 4  # Table 2


@pytest.mark.parametrize("r", SMALL_D, ids=[f"R{r['R']}_D{r['D']}" for r in SMALL_D])
def test_oracle_error_within_the_papers_range(r):
    I1, I2, (tu, tv) = _pair(r)
    u, v = oracle.flow(I1.astype(np.float64), I2.astype(np.float64),
                       oracle.Params(psl=r["psl"], kr=r["kr"], it=r["it"], nr=r["nr"], bits=12))
    err = float(np.hypot(u - tu, v - tv).mean())
    print(f"R={r['R']} D={r['D']}: <Err> = {err:.4f} px")
    assert err <= ERR_RANGE[1]


@pytest.mark.gpu
def test_gpu_error_within_the_papers_range():
    """The CUDA path on every Table 3 case with D <= 16 px (12-bit input,
    NR on, KR up to 6, PSL up to 4), same bound."""
    torch = pytest.importorskip("torch")
    import paper_2509_25924_gb300 as ofv
    dev = torch.device("cuda:0")
    for r in SMALL_D:
        I1, I2, (tu, tv) = _pair(r)
        p = ofv.ofv_default_params(levels_psl=r["psl"], kernel_radius=r["kr"], iterations=r["it"],
                                   norm_radius=r["nr"])
        h = ofv.ofv_create(N, N, p)
        try:
            u = torch.empty((N, N), device=dev); v = torch.empty_like(u)
            ofv.ofv_compute(h, torch.from_numpy(I1).to(dev), torch.from_numpy(I2).to(dev), u, v)
            torch.cuda.synchronize()
            err = float(np.hypot(u.cpu().numpy() - tu, v.cpu().numpy() - tv).mean())
        finally:
            ofv.ofv_destroy(h)
        print(f"GPU R={r['R']} D={r['D']}: <Err> = {err:.4f} px")
        assert err <= ERR_RANGE[1], (r, err)


def test_turbulence_prefers_the_papers_small_kernel():
    """Sec. 5 (HIT): the best parameters for the turbulent case are small
    kernels, KR 2, NR 1, PSL 2, IT 5 with particles of sigma 1 px at 0.119
    particles per pixel, for <Err> = 0.163 px (Table 4).  On the synthetic
    turbulence stand-in (Kolmogorov-like spectrum, rms 2 px; not the DNS),
    the same parameters beat the default KR 4 and land near the paper's
    error (measured 0.193 against 0.260 px)."""
    H = W = 1024
    fld = synth.turbulence_field(H, W, seed=3).sampled(H, W)
    tu, tv = fld.grid(H, W)
    I1, I2 = synth.particle_pair(H, W, fld, ppp=0.119, dmin=2.35, dmax=2.35, seed=3, noise=0.0, bits=12,
                                 kind=synth.OUT_U16, field_max=8.0)
    s = (slice(16, -16), slice(16, -16))

    def err(**p):
        u, v = oracle.flow(I1.astype(np.float64), I2.astype(np.float64), oracle.Params(bits=12, **p))
        return float(np.hypot(u - tu, v - tv)[s].mean())

    best = err(psl=2, kr=2, it=5, nr=1)
    default = err(psl=2, kr=4, it=3, nr=0)
    print(f"turbulence stand-in: paper's HIT parameters {best:.3f} px, default {default:.3f} px")
    assert best < default and best <= 0.25
