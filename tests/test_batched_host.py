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
    names = [n for n, _ in Autotuner.candidates()]
    assert names == ["popc", "tc0", "tc1", "tc2", "tc3"]
