"""C-ABI checks that need no GPU: the library loads, exports every declared function,
has the paper's defaults, sizes workspaces and rejects invalid arguments before any
launch."""
import ctypes
import json
import os

import pytest

from tests._lib import built_lib, header_functions

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


@pytest.fixture(scope="module")
def L():
    return built_lib()


def test_exports_every_declared_function(L):
    names = header_functions()
    assert "mfipm_solve" in names and "mfipm_solve_batched" in names and "mfipm_backward" in names
    for name in names:
        assert hasattr(L, name), name
    from paper_1208_5435_gb300 import _capi
    assert set(_capi.SIGNATURES) == set(names)


def test_param_defaults_are_the_papers(L):
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    assert L.mfipm_params_default(ctypes.byref(p)) == 0
    g = json.load(open(GOLDEN))
    assert (p.sigma1, p.sigma2, p.sigma3) == (g["sigma1"], g["sigma2"], g["sigma3"])
    assert (p.alpha_bar, p.alpha_tilde) == (g["alpha_bar"], g["alpha_tilde"])
    assert p.max_iter == g["maxiters"] and p.max_iter_pcg == g["mxiterpcg"]
    assert g["tolpcg_noisy_range"][0] <= p.tol_pcg <= g["tolpcg_noisy_range"][1]
    assert g["tol_noisy_range"][0] <= p.tol <= g["tol_noisy_range"][1]
    assert L.mfipm_params_default(None) == C.MFIPM_INVALID_ARG


def test_python_params_mirror_the_c_defaults(L):
    """SolverParams() (the binding's defaults) equals mfipm_params_default field by field."""
    import paper_1208_5435_gb300 as M
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    assert L.mfipm_params_default(ctypes.byref(p)) == 0
    q = M.SolverParams().to_c(C.PREC_FP32_PCG)
    for name, _ in C.Params._fields_:
        assert getattr(p, name) == getattr(q, name), name
    assert p.outer_f32_gap == 1e-8
    p.outer_f32_gap = -1.0
    op = _dct_op(C, 1024, 256)
    nb = ctypes.c_size_t()
    ws = ctypes.c_void_p(0x100000)
    info = C.Info()
    assert L.mfipm_solve(ctypes.byref(op), ctypes.c_void_p(0x3000), 0.1, ctypes.byref(p), ctypes.c_void_p(0x4000),
                         None, ws, 1 << 30, ctypes.byref(info), None) == C.MFIPM_INVALID_ARG
    assert b"outer_f32_gap" in L.mfipm_last_error()


def _dct_op(C, n, m, rows_ptr=0x1000):
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = C.OP_PARTIAL_DCT, 0, m, n, None, 1.0, 0, rows_ptr
    return op


def test_workspace_size_grows_with_batch(L):
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    sizes = []
    for batch in (1, 2, 8):
        ops = (C.Operator * batch)(*[_dct_op(C, 4096, 1024) for _ in range(batch)])
        nb = ctypes.c_size_t()
        assert L.mfipm_workspace_size(ops, batch, ctypes.byref(p), ctypes.byref(nb)) == 0
        sizes.append(nb.value)
    assert sizes[0] >= 4096 * 80 and sizes[0] < sizes[1] < sizes[2]


@pytest.mark.parametrize("case", ["n_bad_length", "n_odd", "m_gt_n", "n_too_big", "tau_nonpositive", "null_ws", "small_ws",
                                  "bad_cluster", "bad_eta", "dense_bf16_here", "dct_bf16_prec"])
def test_invalid_arguments_rejected_before_launch(L, case):
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    op = _dct_op(C, 4096, 1024)
    tau = 0.1
    ws, wsb = ctypes.c_void_p(0x10000), 1 << 40
    if case == "n_bad_length":
        op.n = 1400  # n/2 = 700 has the prime factor 7
    elif case == "n_odd":
        op.n = 3001
    elif case == "m_gt_n":
        op.m = 5000
    elif case == "n_too_big":
        op.n, op.m = 1 << 21, 1 << 19
    elif case == "tau_nonpositive":
        tau = 0.0
    elif case == "null_ws":
        ws = None
    elif case == "small_ws":
        wsb = 1024
    elif case == "bad_cluster":
        p.cluster_size = 3
    elif case == "bad_eta":
        p.eta = 1.0
    elif case == "dense_bf16_here":
        op.kind, op.a_dtype, op.A, op.lda, op.rows = C.OP_DENSE, C.A_BF16, 0x2000, op.n, None
    elif case == "dct_bf16_prec":
        p.precision = C.PREC_BF16_A
    info = C.Info()
    rc = L.mfipm_solve(ctypes.byref(op), ctypes.c_void_p(0x3000), tau, ctypes.byref(p), ctypes.c_void_p(0x4000),
                       None, ws, wsb, ctypes.byref(info), None)
    assert rc in (C.MFIPM_INVALID_ARG, C.MFIPM_UNSUPPORTED), (case, rc)
    assert L.mfipm_last_error() and len(L.mfipm_last_error()) > 5


def test_large_dct_workspace_and_threshold(L):
    """n above the cluster solver's 65536 goes to the lockstep multi-pass solver; its
    workspace holds about 130 bytes per index and grows with the group."""
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    sizes = []
    for batch in (1, 4):
        ops = (C.Operator * batch)(*[_dct_op(C, 1 << 20, 1 << 18) for _ in range(batch)])
        nb = ctypes.c_size_t()
        assert L.mfipm_workspace_size(ops, batch, ctypes.byref(p), ctypes.byref(nb)) == 0
        sizes.append(nb.value)
    assert sizes[0] >= (1 << 20) * 120 and sizes[1] > 3 * sizes[0] // 2
    # the threshold hook moves n = 4096 onto the multi-pass path and back
    one = (C.Operator * 1)(_dct_op(C, 4096, 1024))
    nb0, nb1 = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.mfipm_workspace_size(one, 1, ctypes.byref(p), ctypes.byref(nb0)) == 0
    assert L.mfipm_set_large_dct_threshold(512) == C.MFIPM_INVALID_ARG
    assert L.mfipm_set_large_dct_threshold(1024) == 0
    try:
        assert L.mfipm_workspace_size(one, 1, ctypes.byref(p), ctypes.byref(nb1)) == 0
    finally:
        assert L.mfipm_set_large_dct_threshold(1 << 17) == 0
    assert nb1.value != nb0.value


@pytest.mark.parametrize("case", ["small_ws", "null_ws", "fp64_pcg", "n_not_pow2", "backward_no_zs"])
def test_large_dct_rejected_before_launch(L, case):
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    op = _dct_op(C, 1 << 20, 1 << 18)
    ws, wsb = ctypes.c_void_p(0x10000), 1 << 40
    if case == "small_ws":
        wsb = 1 << 20
    elif case == "null_ws":
        ws = None
    elif case == "fp64_pcg":
        p.precision = C.PREC_FP64
    elif case == "n_not_pow2":
        op.n = (1 << 20) - 64
    info = C.Info()
    if case == "backward_no_zs":
        ops = (C.Operator * 1)(op)
        P = ctypes.c_void_p
        arr = (P * 1)(P(0x3000))
        rc = L.mfipm_backward(1, ops, arr, (ctypes.c_double * 1)(0.1), arr, None, arr, None, None, None,
                              ctypes.byref(p), ws, wsb, ctypes.byref(info), None)
    else:
        rc = L.mfipm_solve(ctypes.byref(op), ctypes.c_void_p(0x3000), 0.1, ctypes.byref(p), ctypes.c_void_p(0x4000),
                           None, ws, wsb, ctypes.byref(info), None)
    assert rc in (C.MFIPM_INVALID_ARG, C.MFIPM_UNSUPPORTED), (case, rc)
    assert L.mfipm_last_error() and len(L.mfipm_last_error()) > 5


@pytest.mark.parametrize("fn", ["apply_A", "apply_At", "kkt"])
@pytest.mark.parametrize("case", ["null_vec", "small_ws", "null_ws", "bad_tau"])
def test_operator_products_rejected_before_launch(L, fn, case):
    from paper_1208_5435_gb300 import _capi as C
    op = _dct_op(C, 4096, 1024)
    vin, vout = ctypes.c_void_p(0x3000), ctypes.c_void_p(0x4000)
    ws, wsb, tau = ctypes.c_void_p(0x10000), 1 << 40, 0.1
    if case == "null_vec":
        vin = None
    elif case == "small_ws":
        wsb = 4096
    elif case == "null_ws":
        ws = None
    elif case == "bad_tau":
        if fn != "kkt":
            pytest.skip("tau only enters the KKT residual")
        tau = -1.0
    if fn == "apply_A":
        rc = L.mfipm_apply_A(ctypes.byref(op), vin, vout, ws, wsb, None)
    elif fn == "apply_At":
        rc = L.mfipm_apply_At(ctypes.byref(op), vin, vout, ws, wsb, None)
    else:
        out = ctypes.c_double()
        rc = L.mfipm_kkt_residual(ctypes.byref(op), ctypes.c_void_p(0x5000), tau, vin, ws, wsb, ctypes.byref(out), None)
    assert rc == C.MFIPM_INVALID_ARG, (fn, case, rc)
    assert len(L.mfipm_last_error()) > 5


def test_autotune_rejected_before_launch(L):
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    ops = (C.Operator * 2)(_dct_op(C, 4096, 1024), _dct_op(C, 2048, 512))
    P = ctypes.c_void_p
    arr = (P * 2)(P(0x3000), P(0x3100))
    taus = (ctypes.c_double * 2)(0.1, 0.1)
    t = C.Tuning()
    assert L.mfipm_autotune(2, ops, arr, taus, ctypes.byref(p), arr, None, 1 << 40, None, ctypes.byref(t), None) \
        == C.MFIPM_INVALID_ARG  # no workspace
    assert L.mfipm_autotune(2, ops, arr, taus, ctypes.byref(p), arr, ctypes.c_void_p(0x10000), 4096, None,
                            ctypes.byref(t), None) == C.MFIPM_INVALID_ARG  # small workspace
    assert L.mfipm_autotune(0, ops, arr, taus, ctypes.byref(p), arr, ctypes.c_void_p(0x10000), 1 << 40, None,
                            ctypes.byref(t), None) == C.MFIPM_INVALID_ARG
    assert t.path == 0
    assert L.mfipm_clear_tuning() == 0


@pytest.mark.parametrize("case", ["n_not_pow2", "n_too_big", "n_too_small", "fp64_outer", "bf16_prec", "null_rows",
                                  "backward"])
def test_partial_haar_rejected_before_launch(L, case):
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    op = _dct_op(C, 4096, 1024)
    op.kind = C.OP_PARTIAL_HAAR
    ws, wsb = ctypes.c_void_p(0x10000), 1 << 40
    if case == "n_not_pow2":
        op.n = 3000
    elif case == "n_too_big":
        op.n, op.m = 1 << 17, 1 << 15
    elif case == "n_too_small":
        op.n, op.m = 32, 8
    elif case == "fp64_outer":
        p.outer = 1
    elif case == "bf16_prec":
        p.precision = C.PREC_BF16_A
    elif case == "null_rows":
        op.rows = None
    info = C.Info()
    if case == "backward":
        # the reverse mode runs on the Haar operator, but dL/dA is defined for dense A only
        one = lambda v: (ctypes.c_void_p * 1)(v)
        rc = L.mfipm_backward(1, ctypes.byref(op), one(0x3000), (ctypes.c_double * 1)(0.1), one(0x4000), one(0x5000),
                              one(0x6000), one(0x7000), (ctypes.c_double * 1)(), one(0x8000), ctypes.byref(p), ws,
                              wsb, ctypes.byref(info), None)
        assert rc == C.MFIPM_UNSUPPORTED, rc
    else:
        rc = L.mfipm_solve(ctypes.byref(op), ctypes.c_void_p(0x3000), 0.1, ctypes.byref(p), ctypes.c_void_p(0x4000),
                           None, ws, wsb, ctypes.byref(info), None)
        assert rc in (C.MFIPM_INVALID_ARG, C.MFIPM_UNSUPPORTED), (case, rc)
    assert L.mfipm_last_error() and len(L.mfipm_last_error()) > 5


def test_partial_haar_workspace_matches_dct(L):
    """The Haar operator keeps the DCT's per-problem state (row mask 1 B, scattered b 16 B,
    iterate 32 B, five PCG pairs 40 B, scratch 8 B per index) but needs no twiddle tables."""
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    sizes = {}
    for kind in (C.OP_PARTIAL_DCT, C.OP_PARTIAL_HAAR):
        op = _dct_op(C, 8192, 2048)
        op.kind = kind
        nb = ctypes.c_size_t()
        assert L.mfipm_workspace_size(ctypes.byref(op), 1, ctypes.byref(p), ctypes.byref(nb)) == 0
        sizes[kind] = nb.value
    assert 97 * 8192 <= sizes[C.OP_PARTIAL_HAAR] < sizes[C.OP_PARTIAL_DCT]


def test_general_length_dct_workspace(L):
    """Lengths that are not powers of two (n/2 with prime factors 2, 3, 5 only) are sized like
    the others plus one roots table per distinct n, shared by the problems of that n."""
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))

    def size(ns):
        ops = (C.Operator * len(ns))(*[_dct_op(C, n, n // 4) for n in ns])
        nb = ctypes.c_size_t()
        assert L.mfipm_workspace_size(ops, len(ns), ctypes.byref(p), ctypes.byref(nb)) == 0, L.mfipm_last_error()
        return nb.value

    one = size([1000])
    same = size([1000, 1000]) - one     # a second problem of the same n: no second table
    other = size([1000, 960]) - one     # a smaller n with a table of its own (3 x 480 roots x 40 B)
    assert other > same and other - same >= 3 * 480 * 40 - 2 * 40 * 1000
    for n in (8, 96, 250, 1000, 6000, 16200):
        assert size([n]) > 0


@pytest.mark.parametrize("case", ["too_long", "factor_7", "cluster", "batch_too_long"])
def test_general_length_dct_rejected_before_launch(L, case):
    from paper_1208_5435_gb300 import _capi as C
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    ws, wsb = ctypes.c_void_p(0x10000), 1 << 40
    info = C.Info()
    P = ctypes.c_void_p
    ops = [_dct_op(C, 1000, 250)]
    if case == "too_long":
        ops = [_dct_op(C, 20000, 5000)]   # n/2 = 2^4 5^4, above one CTA's 16384
    elif case == "factor_7":
        ops = [_dct_op(C, 1400, 300)]
    elif case == "cluster":
        p.cluster_size = 4
    elif case == "batch_too_long":
        ops = [_dct_op(C, 1000, 250), _dct_op(C, 32768, 8192)]
    arr = (C.Operator * len(ops))(*ops)
    ptrs = (P * len(ops))(*[P(0x3000)] * len(ops))
    taus = (ctypes.c_double * len(ops))(*[0.1] * len(ops))
    infos = (C.Info * len(ops))()
    rc = L.mfipm_solve_batched(len(ops), arr, ptrs, taus, ctypes.byref(p), ptrs, None, ws, wsb, infos, None)
    assert rc in (C.MFIPM_INVALID_ARG, C.MFIPM_UNSUPPORTED), (case, rc)
    assert len(L.mfipm_last_error()) > 5
