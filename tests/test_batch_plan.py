"""Host logic of the batched form, on the CPU: the pass table lre_batch_run
builds (test hook lre_debug_batch_plan, no device work).  The persistent
kernel relies on it: units are numbered pass-major, each unit's dependency
is the whole previous pass of its own instance and lies at strictly smaller
unit numbers (so the smallest unfinished unit can always run), and every
instance's passes contract all n qubits."""
import ctypes
import os
import subprocess

import pytest

C_FOLD, C_ASM, C_ASM6 = 0, 32, 48
I32, I16 = 0, 1  # lre_count_kind


@pytest.fixture(scope="module")
def lib():
    if subprocess.call(["which", "nvcc"], stdout=subprocess.DEVNULL) != 0 and \
            not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1602_08604_gb300 import build, lre
    build.build()
    L = lre.load()
    f = L.lre_debug_batch_plan
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    f.restype = ctypes.c_int
    return lre, f


def _descs(lre, specs):
    """specs: (n, kind, shots, with_rho); fake, aligned device addresses (never
    dereferenced by the planner)."""
    arr = (lre.lre_instance * len(specs))()
    for k, (n, kind, shots, with_rho) in enumerate(specs):
        base = 0x10000000 * (k + 1)
        arr[k] = lre.lre_instance(base, kind, n, shots, base + 0x4000000, base + 0x8000000 if with_rho else None)
    return arr


def _plan(lib, specs, sched):
    lre, f = lib
    arr = _descs(lre, specs)
    nph = f(ctypes.cast(arr, ctypes.c_void_p), len(arr), *sched, None, 0)
    assert nph > 0
    buf = (ctypes.c_int64 * (8 * nph))()
    assert f(ctypes.cast(arr, ctypes.c_void_p), len(arr), *sched, buf, nph) == nph
    keys = ("inst", "code", "dep", "dep_units", "per_unit", "unit_begin", "units", "items")
    return [dict(zip(keys, buf[8 * k:8 * k + 8])) for k in range(nph)]


SPECS = [(1, I32, 700, True), (2, I16, 500, True), (3, I32, 9000, False), (4, I32, 1234, True),
         (5, I16, 800, True), (6, I32, 2000, True), (7, I16, 1000, True), (8, I32, 640, False),
         (9, I32, 10000, True), (3, I16, 77, True), (6, I16, 3000, False), (9, I16, 1500, True)]
SCHEDULES = [(2, 256, 256), (3, 1024, 1024), (3, 256, 4096), (2, 1024, 1024)]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_units_are_numbered_pass_major_and_contiguous(lib, sched):
    ph = _plan(lib, SPECS, sched)
    u = 0
    level_of, seen = [], {}
    for p in ph:
        assert p["unit_begin"] == u
        assert p["per_unit"] == 1 or p["per_unit"] % 256 == 0
        assert p["units"] == -(-p["items"] // p["per_unit"])
        u += p["units"]
        lvl = seen.get(p["inst"], 0)
        seen[p["inst"]] = lvl + 1
        level_of.append(lvl)
    assert level_of == sorted(level_of)  # the first pass of every instance, then the second, ...
    assert set(seen) == set(range(len(SPECS)))


@pytest.mark.parametrize("sched", SCHEDULES)
def test_every_dependency_is_the_previous_pass_at_smaller_units(lib, sched):
    ph = _plan(lib, SPECS, sched)
    last = {}
    for k, p in enumerate(ph):
        d = p["dep"]
        assert d == last.get(p["inst"], -1)
        if d >= 0:
            q = ph[d]
            assert q["inst"] == p["inst"] and d < k
            assert p["dep_units"] == q["units"]
            assert q["unit_begin"] + q["units"] <= p["unit_begin"]  # waits only on smaller units
        else:
            assert p["dep_units"] == 0
        last[p["inst"]] = k


@pytest.mark.parametrize("sched", SCHEDULES)
def test_passes_contract_every_qubit(lib, sched):
    ph = _plan(lib, SPECS, sched)
    jmax = sched[0]
    for i, (n, kind, shots, with_rho) in enumerate(SPECS):
        mine = [p for p in ph if p["inst"] == i]
        folds = [p for p in mine if p["code"] < C_ASM]
        asm = [p for p in mine if p["code"] >= C_ASM]
        # fold passes: J = (code >> 3) + 1 qubits each, the first reading the
        # counts of this instance's kind, the last (and only the last) final
        js = [((p["code"] - C_FOLD) >> 3) + 1 for p in folds]
        assert sum(js) == n and max(js) <= jmax
        assert js[-1] <= 2  # the final pass contracts at most two qubits
        for k, p in enumerate(folds):
            c = p["code"] - C_FOLD
            assert bool(c & 4) == (k == 0)
            assert bool(c & 1) == (k == len(folds) - 1)
            if k == 0:
                assert bool(c & 2) == (kind == I32)
            else:
                assert c & 2  # later passes read int32 partials
            r = n - sum(js[:k])
            C = 4 ** sum(js[:k])
            assert p["items"] == 3 ** (r - js[k]) * 2 ** (r - js[k]) * C
            assert p["per_unit"] == (sched[1] if k == 0 else sched[2])
        # assembly passes: only with rho; six qubits in one block pass for n >= 6
        if not with_rho:
            assert not asm
            continue
        qubits = 0
        for p in asm:
            if p["code"] >= C_ASM6:
                assert qubits == 0 and n >= 6
                assert p["items"] == 4 ** (n - 6) and p["per_unit"] == 1
                qubits += 6
            else:
                J = ((p["code"] - C_ASM) >> 2) + 1
                assert p["items"] == 4 ** n // 4 ** J
                qubits += J
        assert qubits == n
        assert (asm[-1]["code"] & 1) == 1  # the last writes rho


def test_rejected_descriptors(lib):
    lre, f = lib
    arr = _descs(lre, [(10, I32, 100, True)])  # n above 9
    assert f(ctypes.cast(arr, ctypes.c_void_p), 1, 3, 1024, 1024, None, 0) == -1
    arr = _descs(lre, [(4, I32, 0, True)])  # no shots
    assert f(ctypes.cast(arr, ctypes.c_void_p), 1, 3, 1024, 1024, None, 0) == -1


def test_batched_byte_model_by_hand():
    """bench.py's algorithmic bytes of a batched launch, for shapes worked by
    hand: n = 1 (one final fold pass 6 x 4 B in, theta + T 4 x 16 B out; one
    assembly pass 4 x 8 B in, 4 x 8 B out) and n = 4 at jmax 3 (fold 3 + 1
    qubits; assembly 2 + 2 qubits)."""
    import bench
    assert bench.batched_alg_bytes([1], 3) == 24 + 64 + 32 + 32
    fold4 = (6 ** 4 * 4 + 6 * 64 * 4) + (6 * 64 * 4 + 256 * 16)
    asm4 = (256 * 8 + 256 * 16) + (256 * 16 + 256 * 8)
    assert bench.batched_alg_bytes([4], 3) == fold4 + asm4
    assert bench.batched_alg_bytes([1, 4], 3) == 152 + fold4 + asm4
