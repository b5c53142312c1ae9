"""Mixed precision (FP32-level tensor-core contractions, FP64 Cholesky, rank
decisions and error bookkeeping) and the FP64 path against the FP64 oracle, up to
the banded QTT workload of 2^12 x 2^12 (12 modes of size 4, eps = 1e-6).

At 2^12 the oracle takes about ten minutes, so its result is read from
tests/golden/qtt12_oracle.json (written by tests/golden/make_qtt_golden.py, which
calls only the oracle): ranks, per-bond largest / last kept / first dropped
singular values, the discarded tail and the oracle TT at 1,024 seeded positions
(half of them nonzeros of the input).  The sampled comparison is a necessary
condition of the Frobenius one: every entry of B_gpu - B_oracle is bounded by
||B_gpu - B_oracle||_F.

Bars: ranks equal to the oracle's in both precisions (the mixed path keeps an
FP32-level bond only when its rank decision is resolved, otherwise it redoes
the bond with FP64-level products); products within 1e-12 (FP64) and 1e-5
(mixed) of ||A||_F.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import dense as D
from oracle import fasttt as O
from paper_1908_02721_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5
FP64_TOL = 1e-12
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "qtt12_oracle.json")


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _cores_np(tt):
    return [c.detach().cpu().numpy() for c in tt.cores()]


@pytest.mark.parametrize("name", ["uniform5-n30", "qtt-m10", "qtt-m10-eps1e-3"])
def test_mixed_precision_against_fp64_oracle(F, name):
    if name == "uniform5-n30":
        w = W.uniform5(seed=2, nnz=7776, n=30)
    elif name == "qtt-m10":
        w = W.banded_qtt(10)
    else:
        w = W.banded_qtt(10, eps=1e-3)
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps, precision="mixed")
    res = O.fasttt(w.idx, w.vals, w.dims, w.eps)
    assert tt.stats["p"] == res.p
    assert tt.ranks == res.ranks
    nA = math.sqrt(res.norm2)
    diff = D.tt_diff_norm(_cores_np(tt), res.cores)
    assert diff <= MIXED_TOL * nA, diff / nA
    assert abs(tt.stats["err2"] - res.err2) <= 1e-3 * res.err2 + MIXED_TOL * res.norm2
    tt.free()


def _golden():
    with open(GOLDEN) as f:
        g = json.load(f)
    g["norm2"] = float.fromhex(g["norm2"])
    g["err2"] = float.fromhex(g["err2"])
    g["tt_at_samples"] = np.array([float.fromhex(x) for x in g["tt_at_samples"]])
    return g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_qtt12_against_oracle_golden(F, precision):
    g = _golden()
    w = W.banded_qtt(g["m"], eps=g["eps"])
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps, precision=precision, keep_intermediates=True)
    st = tt.stats
    assert st["p"] == g["p"] and st["R"] == g["R"] and st["rt"] == g["rt"]
    assert tt.ranks == g["ranks"]
    assert abs(st["norm2"] - g["norm2"]) <= 1e-14 * g["norm2"]
    nA = math.sqrt(g["norm2"])
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    for b, info in g["bonds"].items():
        sig = tt.array("sigma", int(b)).cpu().numpy()
        s1 = float.fromhex(info["sigma_first"])
        assert abs(sig[0] - s1) <= tol * nA
        assert abs(sig[info["rank"] - 1] - float.fromhex(info["sigma_last_kept"])) <= tol * nA
    # discarded energy: the dropped singular values sit near delta; FP64 resolves them to
    # u * s1^2 / sigma, the mixed path (which keeps the bond only where resolved) likewise
    assert abs(st["err2"] - g["err2"]) <= 1e-3 * g["err2"] + tol ** 2 * g["norm2"]
    pos = W.sample_positions(w, g["n_samples"] // 2, g["n_samples"] // 2, g["sample_seed"])
    vals = F.tt_eval_at(tt.cores(), torch.from_numpy(pos).cuda()).cpu().numpy()
    assert np.max(np.abs(vals - g["tt_at_samples"])) <= tol * nA
    if precision == "mixed":
        # the per-bond precision choice: the well-conditioned Gram bonds stay at FP32
        # level, the bond whose kept spectrum reaches 1e-6 of sigma_1 is redone at FP64
        assert st["mixed_fp32_bonds"] >= 1 and st["mixed_fp64_bonds"] >= 1
    tt.free()


def test_mixed_never_silently_wrong_at_eps0(F):
    # eps = 0 keeps every numerically nonzero singular value: no FP32-level Gram can
    # decide that, so the mixed path must agree with FP64 (or fail loudly)
    w = W.banded_qtt(9, eps=0.0)
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 0.0, precision="mixed")
    res = O.fasttt(w.idx, w.vals, w.dims, 0.0)
    assert tt.ranks == res.ranks
    nA = math.sqrt(res.norm2)
    assert D.tt_diff_norm(_cores_np(tt), res.cores) <= MIXED_TOL * nA
    tt.free()
