"""The benchmark's exact mixed step against the oracle.

N = 8000 theta solution (400 chains x 20 beads, c/c* = 4, EV off, overlap
correction on), alpha = 2 sqrt(pi)/L (230 half-space k-vectors, K_p = 960 reciprocal
columns on the tensor cores), the symmetric product shape, m = 16 Wiener columns,
N_Ch = 40, lagged bounds with the benchmark's settings.  One direct bd_step
(explicit dW) and one replay of the captured step (dW from the device
Philox counter, regenerated here by the oracle's own Philox), each compared
element by element with oracle.step run at that step's own bounds, at the
mixed-mode bars of the method: 1e-5 on D.F after refinement, 1e-3 on the
Brownian term (max-norm relative).  Sampled rows of the FP32 D against the
oracle's rows at 2e-6.  The oracle's step at this size takes one to two
minutes on the host cores.
"""
import numpy as np
import pytest

import oracle
from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

KW = dict(m=16, n_cheb=40, lanczos_iters=30, bound_safety=0.05, dmin_fraction=0.5,
          bounds_mode=1)


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    oracle.build()
    return binding


def check_step(p, R_in, R_out, dW, st, DF, dS):
    R_ref, code, DF_r, dS_r, _ = oracle.step(p, R_in, dW, st["d_min"], st["d_max"], KW["n_cheb"])
    assert code == 0 and st["accepted"] == 1 and st["status"] == 0
    e = {"DF": relerr(DF, DF_r), "dS": relerr(dS, dS_r),
         "disp": relerr(R_out.reshape(-1) - R_in.reshape(-1),
                        R_ref.reshape(-1) - R_in.reshape(-1))}
    assert e["DF"] <= 1e-5, e
    assert e["dS"] <= 1e-3, e
    assert e["disp"] <= 1e-3, e
    return e


def test_headline_mixed_step_and_replay_vs_oracle(bnd):
    cfg, _ = inputs.preset("c4", alpha_factor=2.0)
    p = cfg.params()
    n3, m = 3 * cfg.n, KW["m"]
    R0 = inputs.make_chains(cfg)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=m, max_cheb=KW["n_cheb"])
    assert plan.info.n_kvec == 230              # K_p = 4 x 230 padded to 960
    plan.set_shape(bnd.BD_SHAPE_SYMMETRIC)
    R = torch.tensor(R0, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    DF = torch.empty(n3, dtype=torch.float64, device="cuda")
    dS = torch.empty(m, n3, dtype=torch.float64, device="cuda")

    # direct step (the first of a lagged run takes fresh bounds)
    dW0 = inputs.make_wiener(n3, m, p["dt"], 501)
    plan.step(R, D, torch.tensor(dW0, device="cuda"), DF=DF, dS=dS, stats=stats, **KW)
    torch.cuda.synchronize()
    st0 = bnd.read_stats(stats)
    # rows of the FP32 D of that step (R0): tiles on and above the diagonal
    # (the symmetric shape leaves the rest of the lower triangle unwritten,
    # so only those columns are read back)
    D32 = plan.D_view(D, "f32")
    for b0 in (0, 3997, 7992):
        rows = oracle.build_D_rows(p, R0, b0, b0 + 8)
        for i in range(24):
            r = 3 * b0 + i
            c0 = (r // 128) * 128
            got = D32[r, c0:].cpu().numpy().astype(np.float64)
            assert relerr(got, rows[i, c0:]) <= 2e-6, (b0, i)
    R1 = R.cpu().numpy().copy()
    e0 = check_step(p, R0, R1, dW0, st0, DF.cpu().numpy(), dS.cpu().numpy())

    # the step captured once and replayed: lagged bounds from the direct step,
    # noise from the device Philox counter
    seed, ctr = 77, 4000
    plan.step_capture(R, D, DF=DF, dS=dS, stats=stats, seed=seed,
                      **{k: v for k, v in KW.items()})
    plan.set_step_counter(ctr)
    plan.step_replay()
    torch.cuda.synchronize()
    st1 = bnd.read_stats(stats)
    dW1 = oracle.wiener_philox(seed, ctr, n3 * m, p["dt"]).reshape(m, n3)
    R2 = R.cpu().numpy().copy()
    e1 = check_step(p, R1, R2, dW1, st1, DF.cpu().numpy(), dS.cpu().numpy())
    # lagged bounds of the replay differ from the fresh ones of the first step
    assert st1["d_max"] != st0["d_max"]
    print("headline step errors vs oracle: direct", e0, "replay", e1)
    plan.close()
