"""Checkpoints on the GPU: a reloaded learned estimator gives the same
estimates, and a reloaded sketch database the same search results."""
import numpy as np
import pytest

from paper_1910_04658_gb300 import checkpoint, inputs
from tests.helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import api, binding as B  # noqa: E402
from paper_1910_04658_gb300 import learned as L  # noqa: E402
from paper_1910_04658_gb300.serving import SketchDB  # noqa: E402


def test_mlp_checkpoint_resume(tmp_path):
    mlp = L.MLPEstimator(seed=2)
    sets = [L.dense_pairs(20_000, 256, pair_seed=5)]
    mlp.train(sets, epochs=1, batch=2048)
    p = str(tmp_path / "mlp.bsck")
    checkpoint.save_mlp(p, mlp)
    again = checkpoint.load_mlp(p)
    assert again.step == mlp.step
    held = L.dense_pairs(5000, 256, pair_seed=6)
    assert torch.equal(mlp.estimate(held), again.estimate(held))
    # training continues from the saved moments and step
    h1 = again.train(sets, epochs=1, batch=2048)
    assert np.isfinite(h1).all() and again.step == 2 * mlp.step


def test_sketch_db_checkpoint(tmp_path):
    c = inputs.random_csr(8, 3000, 200_000, 1, 300)
    rp, col = to_dev(c)
    db = SketchDB(rp, col, c.d, 1024, seed=17)
    p = str(tmp_path / "db.bsck")
    db.save(p)
    db2 = SketchDB.load(p, expect_N=1024, expect_seed=17)
    assert torch.equal(db.sketch, db2.sketch) and torch.equal(db.pc, db2.pc)
    assert torch.equal(db.tiled, db2.tiled)
    q = inputs.random_csr(9, 50, 200_000, 1, 300)
    qrp, qcol = to_dev(q)
    qs, qp = api.sketch(qrp, qcol, q.d, 1024, 17)
    outs = []
    for d in (db, db2):
        s = torch.empty((50, 20), dtype=torch.float32, device="cuda")
        i = torch.empty((50, 20), dtype=torch.int32, device="cuda")
        wsb = B.bs_topk_pretiled_workspace_bytes(50, d.n, 1024, 20)
        ws = torch.empty((wsb,), dtype=torch.uint8, device="cuda")
        B.bs_topk_pretiled(qs, qp, 50, d.tiled, d.pc, d.n, 1024, B.BS_JS, 20, s, i, ws, wsb)
        outs.append((s, i))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    with pytest.raises(checkpoint.CheckpointError):
        SketchDB.load(p, expect_seed=18)
