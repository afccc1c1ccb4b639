"""Autotuner bookkeeping (no GPU)."""
import json

from paper_1910_04658_gb300.batched import Autotuner


def test_autotuner_cache_roundtrip(tmp_path):
    p = tmp_path / "t.json"
    t = Autotuner(cache_path=str(p))
    assert t.table == {}
    key = Autotuner.key("GB300", 4096, 100_000, 50, "js")
    assert key == "GB300|N=4096|log2n=17|k=50|by=js"
    t.table[key] = 2 | (2 << 4)
    t.save()
    assert json.load(open(p)) == {key: 34}
    assert Autotuner(cache_path=str(p)).table == {key: 34}
    cands = Autotuner.candidates()
    assert [n for n, _ in cands] == ["popc"] + [f"tc{c}" for c in range(15)]
    # variant codes: POPC, then TC with configuration bits (c + 1) << 4
    assert cands[0][1] == 1 and [v for _, v in cands[1:]] == [2 | ((c + 1) << 4) for c in range(15)]
