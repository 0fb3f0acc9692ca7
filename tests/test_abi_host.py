"""Host-side checks of the C ABI: the library loads without a GPU, exports every
function include/qe.h declares, and rejects invalid problems before touching
the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

import __graft_entry__ as G
from paper_1809_11134_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qe.h")


@pytest.fixture(scope="module")
def qe():
    G.build()
    from paper_1809_11134_gb300 import qe as Q
    Q.lib()
    return Q


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(qe_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("qe_init", "qe_sample", "qe_eval", "qe_update", "qe_step", "qe_destroy",
                 "qe_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(qe):
    out = subprocess.run(["nm", "-D", "--defined-only", qe.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (qe_\w+)", out))
    assert set(declared_functions()) <= exported
    assert set(qe.EXPORTS) == set(declared_functions())
    lib = qe.lib()
    for name in declared_functions():
        assert getattr(lib, name) is not None


def test_library_info_matches_oracle(qe):
    import oracle
    for n in range(1, 6):
        for lib in (1, 2, 3, 5, 6, 7):
            if n == 1 and not lib & 2:
                continue
            assert qe.qe_library_info(n, lib) == (oracle.num_gates(n, lib),
                                                  oracle.num_regions(n, lib))
    with pytest.raises(qe.QeError):
        qe.qe_library_info(6, 1)


BAD = [
    dict(n=0), dict(n=6), dict(L=0), dict(L=65), dict(P=0), dict(P=(1 << 20) + 1),
    dict(library=16), dict(library=8 | 1), dict(library=1, n=1), dict(topk=1025), dict(topk=5000, P=4096),
    dict(p_mutation=1.5), dict(p_mutation=float("nan")), dict(mutation_range=float("inf")),
    dict(perm=[0, 0, 1, 2, 3, 4, 5, 6]), dict(perm=[8, 1, 2, 3, 4, 5, 6, 7]),
    dict(precision=3), dict(fitness_kind=2), dict(encoding=2), dict(cost_weight=float("nan")),
    dict(shots=65), dict(reserved=1),
]


@pytest.mark.parametrize("bad", BAD)
def test_init_rejects_invalid_problems_without_a_gpu(qe, bad):
    s = W.Search(3, 8, 64, W.LIB_NCV | W.LIB_HT, W.cknot(3))
    for k, v in bad.items():
        setattr(s, k, v)
    p = qe.to_problem(s)
    if "encoding" in bad:
        p.encoding = bad["encoding"]
    if "reserved" in bad:
        p.reserved = bad["reserved"]
    probs = (qe.qe_problem * 1)(p)
    h = C.c_void_p()
    st = qe.lib().qe_init(C.byref(h), probs, 1, None)
    assert st == qe.QE_EINVAL, qe.lib().qe_last_error(None)
    assert h.value is None
    assert qe.lib().qe_last_error(None)


def test_largest_geometry_fits_uint32_segment_ids(qe):
    # 5 qubits with the full library: 25 regions; L = 64; P = 2^20
    g, r = qe.qe_library_info(5, qe.QE_LIB_NCV | qe.QE_LIB_HT | qe.QE_LIB_IDENTITY)
    assert r * 64 * (1 << 20) < (1 << 32)


def test_allocation_failure_is_reported(qe, monkeypatch):
    monkeypatch.setenv("QE_FAULT_ALLOC", "1")
    s = W.Search(3, 8, 64, W.LIB_NCV, W.cknot(3))
    probs = (qe.qe_problem * 1)(qe.to_problem(s))
    h = C.c_void_p()
    assert qe.lib().qe_init(C.byref(h), probs, 1, None) == qe.QE_ENOMEM
    assert b"QE_FAULT_ALLOC" in qe.lib().qe_last_error(None)


def test_null_context_calls_are_rejected(qe):
    L = qe.lib()
    assert L.qe_step(None, 1, None) == qe.QE_EINVAL
    assert L.qe_sample(None, 0, 0, None, None) == qe.QE_EINVAL
    assert L.qe_eval(None, 0, None, 0, None, None, None) == qe.QE_EINVAL
    L.qe_destroy(None)


def test_struct_layouts(qe):
    assert C.sizeof(qe.qe_problem) == 112
    assert qe.qe_problem.shots.offset == 104
    assert C.sizeof(qe.qe_ranked) == 16
    assert C.sizeof(qe.qe_report) == 120 + 512


def test_ising_library_geometry_and_acceptance(qe, monkeypatch):
    """QE_LIB_ISING: n rotation regions plus n(n-1)/2 templates, 3n + n(n-1)/2 gates
    (the oracle's numbers); both encodings pass validation (they reach the
    allocation, failed here on purpose), mixing it with a discrete library does not."""
    import oracle
    for n in range(1, 6):
        g, r = qe.qe_library_info(n, qe.QE_LIB_ISING)
        assert (g, r) == (oracle.num_gates(n, oracle.LIB_ISING),
                          oracle.num_regions(n, oracle.LIB_ISING))
    monkeypatch.setenv("QE_FAULT_ALLOC", "1")
    for enc in (W.ENC_QEQEA, W.ENC_GA):
        s = W.Search(3, 8, 64, W.LIB_ISING, W.cknot(3), encoding=enc)
        probs = (qe.qe_problem * 1)(qe.to_problem(s))
        h = C.c_void_p()
        assert qe.lib().qe_init(C.byref(h), probs, 1, None) == qe.QE_ENOMEM
    s = W.Search(3, 8, 64, W.LIB_ISING | W.LIB_NCV, W.cknot(3), encoding=W.ENC_GA)
    probs = (qe.qe_problem * 1)(qe.to_problem(s))
    assert qe.lib().qe_init(C.byref(C.c_void_p()), probs, 1, None) == qe.QE_EINVAL


def test_static_entry_rejects_bad_arguments_without_a_gpu(qe):
    """qe_eval_rank_static checks its problem on the host before any CUDA call:
    a NULL problem, a target that is not a permutation and an oversized batch
    are QE_EINVAL with a message."""
    s = W.Search(3, 8, 64, W.LIB_NCV | W.LIB_HT, W.cknot(3), precision=W.PREC_FP32)
    L = qe.lib()
    msg = C.create_string_buffer(256)
    assert L.qe_eval_rank_static(None, None, 16, None, None, None, msg, 256) == qe.QE_EINVAL
    assert msg.value
    s.perm = [0, 0, 1, 2, 3, 4, 5, 6]
    p = qe.to_problem(s)
    assert L.qe_eval_rank_static(C.byref(p), None, 16, None, None, None, msg, 256) == qe.QE_EINVAL
    assert b"permutation" in msg.value
    s.perm = W.cknot(3)
    p = qe.to_problem(s)
    assert L.qe_eval_rank_static(C.byref(p), None, 65537, None, None, None, msg, 256) == qe.QE_EINVAL
    assert b"65536" in msg.value


def test_binding_constants_match_the_header(qe):
    """every QE_* integer constant the binding defines has the header's value"""
    import re
    hdr = open(os.path.join(ROOT, "include", "qe.h")).read()
    defines = {m.group(1): int(m.group(2).rstrip("uU"), 0)
               for m in re.finditer(r"#define\s+(QE_[A-Z0-9_]+)\s+(\(?[0-9xXa-fA-F]+[uU]?)", hdr)
               if not m.group(2).startswith("(")}
    checked = 0
    for name, value in defines.items():
        if hasattr(qe, name):
            assert getattr(qe, name) == value, name
            checked += 1
    assert checked >= 5 and "QE_BATCH_SLOTS" in defines


def test_async_batch_entry_points_reject_a_null_context(qe):
    import ctypes as C
    L = qe.lib()
    one = (C.c_uint32 * 1)(0)
    t = C.c_uint64()
    assert L.qe_eval_host_batch_async(None, 1, one, one, None, None, None, C.byref(t)) == \
        qe.QE_EINVAL
    assert L.qe_eval_host_batch_wait(None, 1) == qe.QE_EINVAL
    assert L.qe_eval_host_batch(None, 1, one, one, None, None, None) == qe.QE_EINVAL
