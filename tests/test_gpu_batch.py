"""Batched persistent product (a9) against the oracle, per instance."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,nvec,tol", [(torch.float32, 8, 3e-6), (torch.float64, 1, 1e-12),
                                            (torch.float64, 4, 1e-12)])
def test_batch_matches_oracle(orc, dtype, nvec, tol):
    A = api()
    insts = W.batched_instances(count=12, seed=4, sizes=(8, 10, 12, 14))
    hams, xs, ys, refs = [], [], [], []
    for k, d in enumerate(insts):
        st = orc.enumerate_states(d["N"], d["nup"])
        ham = A.Hamiltonian(A.Basis(d["N"], d["nup"], d["bonds"]), d["J"])
        X = np.stack([orc.rng_normal(10 * k + v, 0, st.size) for v in range(nvec)], axis=1)
        if dtype == torch.float32:
            X = X.astype(np.float32).astype(np.float64)
        refs.append(orc.apply_u1(d["N"], st, d["bonds"], d["J"], X))
        x = torch.from_numpy(X).to(dtype).cuda().contiguous()
        if nvec == 1:
            x = x[:, 0].contiguous()
        hams.append(ham)
        xs.append(x)
        ys.append(torch.empty_like(x))
    for _ in range(2):  # first call tunes and captures, second replays the graph
        for y in ys:
            y.zero_()
        A.batch_apply(hams, xs, ys)
        torch.cuda.synchronize()
        for y, ref in zip(ys, refs):
            assert rel_l2(y.double().cpu().numpy().reshape(ref.shape), ref) <= tol


def test_batch_c4_shapes(orc):
    """C4 workload shape: 64 instances, N in {18..28}, chains and ladders,
    8 FP32 right-hand sides each; sampled rows of each instance checked."""
    A = api()
    insts = W.batched_instances(count=64, seed=4)
    hams, xs, ys = [], [], []
    for k, d in enumerate(insts):
        ham = A.Hamiltonian(A.Basis(d["N"], d["nup"], d["bonds"]), d["J"])
        x = torch.stack([A.random_vector(ham.dim, 1000 * k + v, torch.float64) for v in range(8)], 1)
        hams.append(ham)
        xs.append(x.float().contiguous())
        ys.append(torch.empty_like(xs[-1]))
    A.batch_apply(hams, xs, ys)  # tunes, captures
    for y in ys:
        y.zero_()
    A.batch_apply(hams, xs, ys)  # graph replay
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    # every instance: N >= 24 ones take the eight-vector prefix-block kernel
    for k in range(64):
        d = insts[k]
        rows = rng.integers(0, hams[k].dim, 64)
        for v in (0, 7):
            yo = orc.apply_rows_rng(d["N"], d["nup"], d["bonds"], d["J"], 1000 * k + v, rows)
            assert rel_l2(ys[k][torch.from_numpy(rows).cuda(), v].double().cpu().numpy(), yo) < 5e-6


def test_batch_fused_mixed_and_new_couplings(orc):
    """Eight FP32 columns, large (N = 24, prefix blocks) and small operators in
    the one fused launch; after new couplings on a large and a small operator
    the next call uses them (the captured launch is rebuilt)."""
    A = api()
    insts = W.batched_instances(count=7, seed=9, sizes=(12, 14, 24))
    assert {d["N"] for d in insts} >= {24, 12}
    hams, xs, ys = [], [], []
    for k, d in enumerate(insts):
        ham = A.Hamiltonian(A.Basis(d["N"], d["nup"], d["bonds"]), d["J"])
        x = torch.stack([A.random_vector(ham.dim, 500 * k + v, torch.float64) for v in range(8)], 1)
        hams.append(ham)
        xs.append(x.float().contiguous())
        ys.append(torch.empty_like(xs[-1]))
    rng = np.random.default_rng(2)

    def check(Js):
        for y in ys:
            y.zero_()
        A.batch_apply(hams, xs, ys)
        torch.cuda.synchronize()
        for k, d in enumerate(insts):
            rows = np.unique(np.concatenate([[0, hams[k].dim - 1], rng.integers(0, hams[k].dim, 48)]))
            for v in (0, 3, 7):
                yo = orc.apply_rows_rng(d["N"], d["nup"], d["bonds"], Js[k], 500 * k + v, rows)
                got = ys[k][torch.from_numpy(rows).cuda(), v].double().cpu().numpy()
                assert rel_l2(got, yo) < 5e-6, (k, d["N"], v)

    Js = [d["J"] for d in insts]
    check(Js)
    check(Js)  # graph replay
    big = next(k for k, d in enumerate(insts) if d["N"] == 24)
    small = next(k for k, d in enumerate(insts) if d["N"] < 24)
    for k in (big, small):
        Js[k] = 1.7 * Js[k] - 0.4
        hams[k].set_couplings(Js[k])
    check(Js)
    check(Js)
