"""Host logic of step (i), on the CPU: the fold pass schedule behind
lre_estimate and lre_parity_sums (test hook lre_debug_fold_plan, no device
work).  The kernels trust it for exactness: a partial sum after t qubits
covers at most 3^t bases of at most one row total each, so int32 partials
are safe exactly when 3^t times the row-total bound stays below 2^31."""
import ctypes
import itertools
import os
import subprocess

import pytest

T_I16, T_I32, T_I64, T_F64 = 0, 1, 2, 3
M_STORE, M_FINAL_U, M_FINAL_W, M_PARITY = 0, 1, 2, 3
SIZE = {T_I16: 2, T_I32: 4, T_I64: 8, T_F64: 8}
I32, I16 = 0, 1  # lre_count_kind
INT32_MAX = 2 ** 31 - 1


@pytest.fixture(scope="module")
def plan_fn():
    if subprocess.call(["which", "nvcc"], stdout=subprocess.DEVNULL) != 0 and \
            not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1602_08604_gb300 import build, lre
    build.build()
    f = lre.load().lre_debug_fold_plan
    f.argtypes = [ctypes.c_int] * 4 + [ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    f.restype = ctypes.c_int

    def plan(n, kind, weighted, parity, bound, aligned, variant):
        k = f(n, kind, weighted, parity, bound, aligned, variant, None, 0)
        assert k > 0
        buf = (ctypes.c_int64 * (9 * k))()
        assert f(n, kind, weighted, parity, bound, aligned, variant, buf, k) == k
        keys = ("first6", "fused9", "J", "r", "in_t", "acc_t", "mode", "C", "out_bytes")
        return [dict(zip(keys, buf[9 * i:9 * i + 9])) for i in range(k)]
    return plan


def fits32(t, bound):
    return bound > 0 and 3 ** t * bound < INT32_MAX


CASES = [c for c in itertools.product(range(1, 15), (I32, I16), (0, 1), (0, 1),
                                      (0, 1, 44, 1000, 2047, 100000, 2 ** 31 // 3 ** 6, 2 ** 31 // 3 ** 6 + 1),
                                      (0, 1), (0, 1, 2, 256, 258))
         if not (c[2] and c[3])]  # parity sums are unweighted
RAW_TENSOR = 256  # variant flag: the raw tensor-core first pass runs (seven qubits may be folded)


def test_every_schedule_is_exact_and_complete(plan_fn):
    for n, kind, weighted, parity, bound, aligned, variant in CASES:
        ps = plan_fn(n, kind, weighted, parity, bound, aligned, variant)
        where = (n, kind, weighted, parity, bound, aligned, variant)
        t, C, in_t = 0, 1, (T_I16 if kind == I16 else T_I32)
        for k, p in enumerate(ps):
            last = k == len(ps) - 1
            assert p["r"] == n - t and p["C"] == C and p["in_t"] == in_t, where
            t += p["J"]
            # the kind of the first pass, and only the first
            if p["fused9"]:
                assert k == 0 and p["J"] == 9 and p["first6"], where
            elif p["first6"]:
                assert k == 0 and p["J"] in (6, 7), where
            else:
                assert 1 <= p["J"] <= (2 if weighted else 3), where
            # partial-sum type: FP64 when weighted; otherwise int32 exactly
            # when 3^t (row total bound) fits, else int64
            if weighted:
                assert p["acc_t"] == T_F64, where
            else:
                assert p["acc_t"] == (T_I32 if fits32(t, bound) else T_I64), where
            # the last pass divides (or stores parity sums); the others store
            mode = (M_PARITY if parity else M_FINAL_W if weighted else M_FINAL_U) if last else M_STORE
            assert p["mode"] == mode, where
            out = 0 if last else 6 ** (n - t) * 4 ** p["J"] * C * SIZE[p["acc_t"]]
            assert p["out_bytes"] == out, where
            C *= 4 ** p["J"]
            in_t = p["acc_t"]
        assert t == n, where


def test_first_pass_choice(plan_fn):
    for n, kind, weighted, parity, bound, aligned, variant in CASES:
        p = plan_fn(n, kind, weighted, parity, bound, aligned, variant)[0]
        where = (n, kind, weighted, parity, bound, aligned, variant)
        fused = not weighted and n > 9 and aligned and fits32(9, bound) and (variant & 255) >= 2
        seven = (bool(variant & RAW_TENSOR) and kind == I16 and not weighted and n > 7 and aligned
                 and fits32(7, bound) and not fused)
        six = not weighted and n > 6 and aligned and fits32(6, bound) and not fused and not seven
        assert bool(p["fused9"]) == fused, where
        assert bool(p["first6"]) == (fused or seven or six), where
        assert p["J"] == (9 if fused else 7 if seven else 6 if six else p["J"]), where


def test_seven_qubit_first_pass_shrinks_every_buffer_at_n14(plan_fn):
    # the headline shape: int16 counts, 1000 shots, the raw tensor-core pass
    p6 = plan_fn(14, I16, 0, 0, 1000, 1, 0)
    p7 = plan_fn(14, I16, 0, 0, 1000, 1, RAW_TENSOR)
    assert [p["J"] for p in p6] == [6, 3, 3, 2]
    assert [p["J"] for p in p7] == [7, 3, 3, 1]
    assert p7[0]["out_bytes"] == 6 ** 7 * 4 ** 7 * 4
    # each stored intermediate is two thirds of the six-qubit schedule's
    for a, b in zip(p6[:-1], p7[:-1]):
        assert 3 * b["out_bytes"] == 2 * a["out_bytes"]


def test_out_of_range_n(plan_fn):
    from paper_1602_08604_gb300 import lre
    f = lre.load().lre_debug_fold_plan
    assert f(0, I32, 0, 0, 1000, 1, 0, None, 0) == -1
    assert f(15, I32, 0, 0, 1000, 1, 0, None, 0) == -1
