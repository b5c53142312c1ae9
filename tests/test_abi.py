"""The C-ABI library builds, loads and exports every function include/fasttt.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "fasttt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_02721_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fasttt_decompose", "tt_eval_at", "tt_eval_backward", "fasttt_tt_free",
                     "fasttt_tt_ranks", "fasttt_tt_core", "fasttt_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_loads_and_matches_exports(lib):
    from paper_1908_02721_gb300 import fasttt as F
    assert sorted(F.EXPORTS) == _declared()
    assert "sm_103a" in F.version()
    o = F.Opts()
    F._lib.fasttt_default_opts(ctypes.byref(o))
    assert o.p == 0 and o.depar_values == 1 and o.max_rank == 0


def _struct_fields(name):
    """Field names of `typedef struct name {...} name;` in the header, in order."""
    txt = open(os.path.join(ROOT, "include", "fasttt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), txt, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)
        first, *rest = [d.strip() for d in decl.split(",")]
        out.append(first.split()[-1])
        out.extend(rest)
    return out


def test_struct_field_order_matches_header(lib):
    from paper_1908_02721_gb300 import fasttt as F
    assert [f[0] for f in F.Opts._fields_] == _struct_fields("fasttt_opts")
    assert [f[0] for f in F.Stats._fields_] == _struct_fields("fasttt_stats")


def test_struct_layouts_match_header(lib):
    from paper_1908_02721_gb300 import fasttt as F
    # fasttt_opts: six ints, two int64, two ints, one int64; fasttt_stats ends with the
    # route counters (int64)
    assert ctypes.sizeof(F.Opts) == 8 * 4 + 3 * 8
    assert F.Opts.sparse_sweep.offset == 6 * 4 + 2 * 8
    assert F.Opts.max_spin.offset == 8 * 4 + 2 * 8
    assert F.Stats.flop_gemm_oz.offset + 8 == F.Stats.ms_tridiag32.offset
    assert F.Stats.wait_timeouts.offset + 8 == ctypes.sizeof(F.Stats)


def test_calls_without_gpu_fail_loudly(lib):
    import torch
    from paper_1908_02721_gb300 import fasttt as F
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(F.FastTTError):
        F.fasttt_decompose([[0, 1], [1, 0]], [1.0, 2.0], [2, 2], 0.0)


def test_tt_arithmetic_and_fitting_fail_loudly_without_gpu(lib):
    """The entry points added for TT arithmetic and fitting have no CPU path either:
    the binding refuses before the call and the library itself rejects bad
    arguments or reports the missing device."""
    import torch
    from paper_1908_02721_gb300 import fasttt as F
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cores = [torch.zeros((1, 2, 1), dtype=torch.float64)]
    for call in (lambda: F.tt_round(cores, 0.1), lambda: F.tt_add(cores, cores),
                 lambda: F.tt_fit_gd(cores, [[0]], [1.0], 1, 0.1)):
        with pytest.raises(F.FastTTError) as e:
            call()
        assert e.value.code == F.ECUDA
    # straight through the C ABI: argument checks run first, then no device
    out = ctypes.c_void_p(0)
    dims = (ctypes.c_int64 * 1)(2)
    bad_ranks = (ctypes.c_int64 * 2)(2, 1)
    ptrs = (ctypes.c_void_p * 1)(None)
    assert lib.fasttt_tt_round(1, dims, bad_ranks, ptrs, ctypes.c_double(0.1), None, None,
                               ctypes.byref(out), None) == F.EINVAL
    losses = (ctypes.c_double * 2)()
    assert lib.tt_fit_gd(0, dims, bad_ranks, ptrs, 0, ctypes.c_int64(0), None, None, ctypes.c_int64(1),
                         ctypes.c_double(0.1), losses, None) == F.EINVAL


def test_eval_and_adjoint_arguments_rejected_before_any_launch(lib):
    """tt_eval_at, tt_eval_backward and tt_eval_backward_noalloc check the shapes the
    kernels index with (idx (d, m), grad_out (m,), one gradient core per core of its
    core's shape, dtype and device) before the call: a wrong shape is EINVAL, never an
    out-of-bounds device access.  The checks need no GPU."""
    import torch
    from paper_1908_02721_gb300 import fasttt as F
    cores = [torch.zeros((1, 3, 2), dtype=torch.float64), torch.zeros((2, 4, 1), dtype=torch.float64)]
    idx = torch.zeros((2, 5), dtype=torch.int32)
    g = torch.zeros(5, dtype=torch.float64)
    grads = [torch.zeros_like(c) for c in cores]
    bad = [
        lambda: F.tt_eval_at(cores, torch.zeros((3, 5), dtype=torch.int32)),           # idx rows != d
        lambda: F.tt_eval_at(cores, torch.zeros(5, dtype=torch.int32)),                # idx not 2-D
        lambda: F.tt_eval_at([cores[0], torch.zeros((3, 4, 1), dtype=torch.float64)], idx),  # ranks disagree
        lambda: F.tt_eval_backward(cores, idx, torch.zeros(4, dtype=torch.float64)),   # grad_out length
        lambda: F.tt_eval_backward(cores, idx, g, [grads[0]]),                         # one gradient short
        lambda: F.tt_eval_backward_noalloc(cores, idx, g, [grads[0], torch.zeros((2, 4, 2), dtype=torch.float64)]),
        lambda: F.tt_eval_backward_noalloc(cores, idx, g, [grads[0], grads[1].float()]),   # dtype
        lambda: F.tt_eval_backward_noalloc(cores, idx, torch.zeros((5, 1), dtype=torch.float64), grads),
        lambda: F.tt_eval_backward_noalloc(cores, torch.zeros((1, 5), dtype=torch.int32), g, grads),
    ]
    for call in bad:
        with pytest.raises(F.FastTTError) as e:
            call()
        assert e.value.code == F.EINVAL, str(e.value)
    if not torch.cuda.is_available():   # well-formed arguments get as far as the missing device
        for call in (lambda: F.tt_eval_at(cores, idx), lambda: F.tt_eval_backward(cores, idx, g),
                     lambda: F.tt_eval_backward_noalloc(cores, idx, g, grads)):
            with pytest.raises(F.FastTTError) as e:
                call()
            assert e.value.code == F.ECUDA
