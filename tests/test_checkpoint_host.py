"""Checkpoint files without a GPU: qe_checkpoint_info reads a file written by
hand in the documented layout (header, problems, records, per-search states)
and rejects every damaged variant; save/load refuse a null context."""
import ctypes as C
import struct

import numpy as np
import pytest

from paper_1809_11134_gb300 import workloads as W


@pytest.fixture(scope="module")
def qe():
    import __graft_entry__ as G
    G.build()
    from paper_1809_11134_gb300 import qe as Q
    return Q


def fnv1a64(b):
    h = 14695981039346656037
    for x in b:
        h = ((h ^ x) * 1099511628211) & (2**64 - 1)
    return h


def write_ckpt(qe, path, searches, gen, magic=b"QECKPT1\0", version=1, damage=None):
    probs = [qe.to_problem(s) for s in searches]
    pay = b"".join(bytes(p) for p in probs)
    for _ in probs:
        r = qe.qe_report()
        r.generation = gen
        pay += bytes(r)
    for s in probs:
        nb = s.population * s.circuit_len  # a GA genome of zeros
        pay += struct.pack("<Q", nb) + bytes(nb)
    h = fnv1a64(pay)
    if damage == "flip":
        pay = pay[:10] + bytes([pay[10] ^ 1]) + pay[11:]
    if damage == "truncate":
        pay = pay[:-3]
    hdr = magic + struct.pack("<6I2Q", version, len(probs), gen, C.sizeof(qe.qe_problem),
                              C.sizeof(qe.qe_report), 0, len(pay) + (3 if damage == "truncate"
                                                                    else 0), h)
    assert len(hdr) == 48
    open(path, "wb").write(hdr + pay + (b"x" if damage == "trailing" else b""))


def searches():
    return [W.Search(3, 8, 40, W.LIB_NCV | W.LIB_HT, W.cknot(3), seed=4, encoding=W.ENC_GA),
            W.Search(2, 3, 16, W.LIB_ISING, W.cknot(2), seed=9, topk=3, encoding=W.ENC_GA)]


def test_info_reads_the_documented_layout(qe, tmp_path):
    path = str(tmp_path / "a.qeckpt")
    ss = searches()
    write_ckpt(qe, path, ss, 17)
    probs, gen = qe.checkpoint_info(path)
    assert gen == 17 and len(probs) == 2
    for p, s in zip(probs, ss):
        assert bytes(p) == bytes(qe.to_problem(s))


@pytest.mark.parametrize("kind", ["flip", "truncate", "trailing", "magic", "version"])
def test_info_rejects_damaged_files(qe, tmp_path, kind):
    path = str(tmp_path / "b.qeckpt")
    kw = {"damage": kind} if kind in ("flip", "truncate", "trailing") else {}
    if kind == "magic":
        kw["magic"] = b"QECKPT2\0"
    if kind == "version":
        kw["version"] = 2
    write_ckpt(qe, path, searches(), 3, **kw)
    with pytest.raises(qe.QeError) as e:
        qe.checkpoint_info(path)
    assert e.value.status == qe.QE_EINVAL


def test_missing_file_and_null_context(qe, tmp_path):
    with pytest.raises(qe.QeError) as e:
        qe.checkpoint_info(str(tmp_path / "none.qeckpt"))
    assert e.value.status == qe.QE_EIO
    assert qe.lib().qe_save(None, b"x") == qe.QE_EINVAL
    assert qe.lib().qe_load(None, b"x") == qe.QE_EINVAL
