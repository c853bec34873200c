"""Argument checks of the binding (paper_2310_12000_gb300/_lib.py). The C ABI takes bare
pointers, so the binding refuses arrays of the wrong length or shape before the library could
read or write past their ends, and passes correct ones (numpy or torch) through. Runs without
a GPU: the handles sit on a stand-in context whose library accepts every call."""
import ctypes as C

import numpy as np
import pytest

from paper_2310_12000_gb300 import _lib


class _AcceptAll:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            if name == "vl_find_mode":
                args[-1]._obj.value = 1            # a non-null state handle
            return 0
        return call


class _Ctx:
    def __init__(self):
        self.lib = _AcceptAll()
        self.h = None

    def check(self, status):
        assert status == 0


@pytest.fixture
def fac():
    ctx = _Ctx()
    f = _lib.Factor(ctx, C.c_void_p(1), 10, 3)
    yield f
    f.h = None


def test_wrong_lengths_are_refused_before_any_call(fac):
    lib = fac.ctx.lib
    with pytest.raises(ValueError, match="y"):
        fac.find_mode(0, np.zeros(9))
    with pytest.raises(ValueError, match="F"):
        fac.find_mode(0, np.zeros(10), np.zeros(11))
    with pytest.raises(ValueError, match="mode_out"):
        fac.find_mode(0, np.zeros(10), None, None, mode_out=np.zeros(3))
    assert "vl_find_mode" not in lib.calls
    st = fac.find_mode(0, np.zeros(10))
    with pytest.raises(ValueError, match="test_locs"):
        st.pred_var(np.zeros(8))
    with pytest.raises(ValueError, match="Fp"):
        st.pred_var(np.zeros((4, 2)), np.zeros(5))
    with pytest.raises(ValueError, match="var_out"):
        st.pred_var(np.zeros((4, 2)), None, None, np.zeros(4), np.zeros(2))
    with pytest.raises(ValueError, match="X"):
        st.apply(0, np.zeros((9, 2)))
    with pytest.raises(ValueError, match="RHS"):
        st.pcg_solve(np.zeros(11))
    assert "vl_pred_var" not in lib.calls and "vl_apply" not in lib.calls and "vl_pcg_solve" not in lib.calls
    st.h = None


def test_correct_arguments_pass(fac):
    torch = pytest.importorskip("torch")
    lib = fac.ctx.lib
    st = fac.find_mode(0, np.zeros(10), np.zeros(10), None, mode_out=np.zeros(10))
    st2 = fac.find_mode(1, torch.zeros(10, dtype=torch.float64), torch.zeros(10, dtype=torch.float64),
                        None, mode_out=torch.zeros(10, dtype=torch.float64))
    mean, var = st.pred_var(np.zeros((4, 2)), np.zeros(4))
    assert mean.shape == (4,) and var.shape == (4,)
    assert st.apply(0, np.zeros(10)).shape == (10, 1)
    assert st.pcg_solve(np.zeros((10, 3)))[0].shape == (10, 3)
    st.apply_A_noalloc(torch.zeros(10, 2, dtype=torch.float64), torch.zeros(10, 2, dtype=torch.float64))
    with pytest.raises(ValueError, match="Y"):
        st.apply_A_noalloc(torch.zeros(10, 2, dtype=torch.float64), torch.zeros(10, dtype=torch.float64))
    assert lib.calls.count("vl_find_mode") == 2 and "vl_pred_var" in lib.calls
    st.h = st2.h = None


def test_context_calls_check_locations():
    ctx = _Ctx()
    ctx.build_factor = _lib.Context.build_factor.__get__(ctx)
    ctx.knn_prev = _lib.Context.knn_prev.__get__(ctx)
    ctx.knn_cross = _lib.Context.knn_cross.__get__(ctx)
    with pytest.raises(ValueError, match="locs"):
        ctx.build_factor(np.zeros(10), None, 0, 1.0, 0.1, 3)
    with pytest.raises(ValueError, match="order"):
        ctx.build_factor(np.zeros((10, 2)), np.arange(9, dtype=np.int32), 0, 1.0, 0.1, 3)
    bad = np.arange(10, dtype=np.int32)
    bad[3] = 4                                       # a duplicate
    with pytest.raises(ValueError, match="permutation"):
        ctx.build_factor(np.zeros((10, 2)), bad, 0, 1.0, 0.1, 3)
    bad[3] = 10                                      # out of range
    with pytest.raises(ValueError, match="permutation"):
        ctx.build_factor(np.zeros((10, 2)), bad, 0, 1.0, 0.1, 3)
    with pytest.raises(ValueError, match="out"):
        ctx.knn_prev(np.zeros((10, 2)), 3, out=np.zeros((10, 2), np.int32))
    with pytest.raises(ValueError, match="test"):
        ctx.knn_cross(np.zeros((10, 2)), np.zeros((4, 3)), 3)
    assert ctx.lib.calls == []
    assert ctx.knn_prev(np.zeros((10, 2)), 3).shape == (10, 3)
    assert ctx.knn_cross(np.zeros((10, 2)), np.zeros((4, 2)), 3).shape == (4, 3)
    f = ctx.build_factor(np.zeros((10, 2)), np.random.default_rng(0).permutation(10).astype(np.int32),
                         0, 1.0, 0.1, 3)
    f.h = None


@pytest.fixture
def batch():
    ctx = _Ctx()
    b = _lib.Batch.__new__(_lib.Batch)
    b.ctx, b.factors, b.h = ctx, [], C.c_void_p(1)
    b.sizes = [10, 4]
    b.offsets = np.array([0, 10, 14], np.int64)
    yield b
    b.h = None


def test_batch_arguments_are_checked_per_problem(batch):
    lib = batch.ctx.lib
    with pytest.raises(ValueError, match="expected 2 problems"):
        batch.find_mode([0], [np.zeros(10)])
    with pytest.raises(ValueError, match=r"y\[1\]"):
        batch.find_mode([0, 0], [np.zeros(10), np.zeros(5)])
    with pytest.raises(ValueError, match=r"F\[0\]"):
        batch.find_mode([0, 0], [np.zeros(10), np.zeros(4)], [np.zeros(9), np.zeros(4)])
    with pytest.raises(ValueError, match="expected 2 problems"):
        batch.pred_var([np.zeros((3, 2))])
    with pytest.raises(ValueError, match=r"test_locs\[1\]"):
        batch.pred_var([np.zeros((3, 2)), np.zeros(6)])
    with pytest.raises(ValueError, match=r"Fp\[1\]"):
        batch.pred_var([np.zeros((3, 2)), np.zeros((2, 2))], [np.zeros(3), np.zeros(5)])
    assert "vl_batch_find_mode" not in lib.calls and "vl_batch_pred_var" not in lib.calls
    modes = batch.find_mode([0, 0], [np.zeros(10), np.zeros(4)])
    assert [len(v) for v in modes] == [10, 4]
    means, vars_ = batch.pred_var([np.zeros((3, 2)), np.zeros((0, 2))], [np.zeros(3), np.zeros(0)])
    assert [len(v) for v in means] == [3, 0] and [len(v) for v in vars_] == [3, 0]
    assert lib.calls.count("vl_batch_find_mode") == 1 and lib.calls.count("vl_batch_pred_var") == 1
