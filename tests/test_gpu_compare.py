"""The QEQEA-vs-GA comparison on the Ising library (the functions of the
paper's Table 3) runs both encodings in one context and reports consistent
records: accuracies in [0, 1], the generation of the best inside the run, and
threshold generations ordered like the thresholds."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def compare():
    import __graft_entry__ as G
    G.build()
    from paper_1809_11134_gb300 import compare as C
    return C


def test_small_comparison_is_consistent(compare):
    res = compare.run(generations=60, P=128, seed=3)
    rows = res["searches"]
    assert len(rows) == 8 and res["seconds_per_generation"] > 0
    for name, row in rows.items():
        assert 0.0 <= row["best"] <= 1.0 + 1e-12, name
        assert 0 <= row["best_gen"] < 60
        firsts = [row["first"][t] for t in compare.THRESHOLDS if t in row["first"]]
        assert firsts == sorted(firsts)
        assert all(t <= row["best"] for t in row["first"])
    assert "| CNOT | GA |" in compare.table(res)
