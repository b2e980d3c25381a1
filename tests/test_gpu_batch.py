"""Batched replicas (bd_batch_*): uneven N, one plan per replica, one graph
launch per step after the first two calls; mixed replicas with few Wiener
columns run their Chebyshev loops together in one persistent launch.

The replicas advanced by the batch must be bitwise the replicas advanced one
plan at a time with the same options and launch shape (every sum of the
batched loop is taken in an order fixed by the row alone);
the mixed batch is checked against the FP64 oracle; the autotuner keeps a
valid split and the product stays within the mixed tolerance.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def small_batch(count=4):
    return inputs.batch_systems(count=count, seed=7, n_min=40, n_max=260)


@pytest.mark.parametrize("prec", ["fp64", "mixed_f16"])
def test_batch_equals_single_plans(bnd, prec):
    cfgs = small_batch()
    plist = [c.params() for c in cfgs]
    Rs = [inputs.make_chains(c) for c in cfgs]
    kw = dict(m=2, n_cheb=16, lanczos_iters=20, bound_safety=0.05, dmin_fraction=0.5,
              seed=11, step_index=3, bounds_mode=1)
    b = bnd.Batch(plist, prec, max_rhs=2, max_cheb=16)
    Rp = torch.tensor(np.concatenate([r.reshape(-1) for r in Rs]), device="cuda")
    Db = b.alloc_D()
    stats = torch.zeros(b.count * bnd.STATS_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(3):                      # direct, record + launch, replay
        b.step(Rp, Db, stats=stats, **kw)
    torch.cuda.synchronize()
    for i, (p, R) in enumerate(zip(plist, Rs)):
        plan = bnd.Plan(p, prec, max_rhs=2, max_cheb=16)
        if prec != "fp64":
            plan.set_shape(5)      # the batch's shape: its Chebyshev loops run in one launch
        plan.set_step_counter(kw["step_index"])
        D = plan.alloc_D()
        Rg = torch.tensor(R, device="cuda")
        ki = dict(kw, seed=kw["seed"] + i, flags=bnd.BD_STEP_DEVICE_COUNTER)
        for _ in range(3):
            plan.step(Rg, D, None, **ki)
        got = Rp[b.r_off[i]:b.r_off[i] + b.n3[i]]
        assert torch.equal(got, Rg.view(-1)), f"replica {i}"
        assert not torch.equal(Rg.view(-1), torch.tensor(R.reshape(-1), device="cuda"))
    st = [bnd.BdStepStats.from_buffer_copy(bytes(stats[i * bnd.STATS_BYTES:(i + 1) * bnd.STATS_BYTES]
                                                 .cpu().numpy().tobytes()))
          for i in range(b.count)]
    assert all(s.accepted == 1 and s.status == 0 for s in st)


def test_batch_mixed_step_vs_oracle(bnd):
    """One batched mixed step: each replica's displacement against the FP64
    oracle step with the same Philox noise and the bounds the replica used."""
    cfgs = small_batch(3)
    plist = [c.params() for c in cfgs]
    Rs = [inputs.make_chains(c) for c in cfgs]
    b = bnd.Batch(plist, "mixed_f16", max_rhs=1, max_cheb=24)
    Rp = torch.tensor(np.concatenate([r.reshape(-1) for r in Rs]), device="cuda")
    Db = b.alloc_D()
    stats = torch.zeros(b.count * bnd.STATS_BYTES, dtype=torch.uint8, device="cuda")
    b.step(Rp, Db, m=1, n_cheb=24, lanczos_iters=40, seed=21, step_index=9, stats=stats,
           bounds_mode=0)
    torch.cuda.synchronize()
    for i, (p, R) in enumerate(zip(plist, Rs)):
        s = bnd.BdStepStats.from_buffer_copy(
            bytes(stats[i * bnd.STATS_BYTES:(i + 1) * bnd.STATS_BYTES].cpu().numpy().tobytes()))
        dW = oracle.wiener_philox(21 + i, 9, 3 * len(R), p["dt"]).reshape(1, -1)
        R_ref, code, *_ = oracle.step(p, R, dW, s.d_min, s.d_max, 24)
        assert code == 0
        disp = Rp[b.r_off[i]:b.r_off[i] + b.n3[i]].cpu().numpy() - R.reshape(-1)
        ref = R_ref.reshape(-1) - R.reshape(-1)
        assert np.max(np.abs(disp - ref)) <= 1e-3 * np.max(np.abs(ref))


def test_autotune_split(bnd):
    cfg = inputs.SystemConfig(n_chains=60, nb=10, c_over_cstar=2.0, seed=5)
    p = cfg.params()
    plan = bnd.Plan(p, "mixed_f16", max_rhs=16)
    R = inputs.make_chains(cfg)
    D = plan.alloc_D()
    plan.build_D(torch.tensor(R, device="cuda"), D)
    split, ms = plan.autotune(D)
    assert split in (1, 2, 3) and ms > 0
    X = inputs.make_wiener(3 * cfg.n, 16, 1.0, 6)
    Y = torch.empty(16, 3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.apply(D, torch.tensor(X, device="cuda"), Y)
    ref = oracle.apply_D(oracle.build_D(p, R), X)
    assert np.max(np.abs(Y.cpu().numpy() - ref)) <= 2e-3 * np.max(np.abs(ref))
