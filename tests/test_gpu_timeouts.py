"""Bounded device waits that run out, and the library afterwards.

Every device spin-wait is bounded: the grid barriers of the cooperative kernels
(Jacobi sweeps, tridiagonalisation) and the tensor-core GEMM's pipeline waits.
With opts.max_spin > 0 a wait that exhausts that many polls sets a device flag,
the kernel leaves (the GEMM only after its copies and MMAs in flight have
completed), and the call fails with FASTTT_ETIMEOUT; the host-side Jacobi sweep
bound (max_sweeps) fails the same way.  After either, the same process must run
a normal decomposition to the oracle's result.  No GPU fault is involved: the
waits give up on purpose, on flags that are set late.
"""
import math

import numpy as np
import pytest

from oracle import dense as D
from oracle import fasttt as O
from paper_1908_02721_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _normal_call_matches_oracle(F, w):
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps)
    res = O.fasttt(w.idx, w.vals, w.dims, w.eps)
    assert tt.ranks == res.ranks
    cores = [c.cpu().numpy() for c in tt.cores()]
    assert D.tt_diff_norm(cores, res.cores) <= 1e-12 * math.sqrt(res.norm2)
    assert tt.stats["wait_timeouts"] == 0
    tt.free()


@pytest.mark.parametrize("engine", ["tensor", "dfma"])
def test_max_spin_waits_give_up_with_etimeout(F, engine):
    # 30^5, 7,776 nonzeros: Gram-route SVDs (tensor-core Grams with engine "tensor"),
    # cooperative Jacobi sweeps and the FP32 tridiagonalisation all wait on the device
    w = W.uniform5(seed=2, nnz=7776, n=30)
    with pytest.raises(F.FastTTError) as e:
        F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps, gemm_engine=engine, max_spin=1)
    assert e.value.code == F.ETIMEOUT, str(e.value)
    assert e.value.stats is not None and e.value.stats["wait_timeouts"] >= 1
    _normal_call_matches_oracle(F, w)


def test_jacobi_sweep_bound_gives_etimeout(F):
    w = W.exact_small()
    with pytest.raises(F.FastTTError) as e:
        F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps, max_sweeps=1)
    assert e.value.code == F.ETIMEOUT, str(e.value)
    _normal_call_matches_oracle(F, w)


def test_generous_max_spin_changes_nothing(F):
    w = W.exact_small()
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps, max_spin=1 << 30)
    res = O.fasttt(w.idx, w.vals, w.dims, w.eps)
    assert tt.ranks == res.ranks and tt.stats["wait_timeouts"] == 0
    tt.free()
