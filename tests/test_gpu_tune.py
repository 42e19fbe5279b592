"""The autotuner (tune.py): it times launch-shape candidates on the GPU, writes
a table, and handles set up with that table take its choices.  The choices
change launch shapes only, so the tuned build still matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk, tune  # noqa: E402


def test_tuned_table_is_used_and_matches_oracle(tmp_path):
    path = str(tmp_path / "tune.txt")
    rows = tune.tune(path, buckets=[(0, 150, 6), (150, 300, 14)], reps=1)
    assert len(rows) == 2 and all(r[-1] > 0 for r in rows)
    for lo, hi, natom in [(0, 150, 6), (150, 300, 14)]:
        m = I.molecule(natom, seed=1000 + natom)
        h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED, tune_table=path)
        row = next(r for r in rows if r[0] <= m.nao < r[1])
        assert h.tuning == row[2:6]
        S = O.overlap(m.orb, m.coords)
        C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000), S)
        ref = O.dfjk(m.orb, m.aux, m.coords, C)
        J, K, EJ, EK = h.build(torch.from_numpy(C).cuda())
        assert np.abs(J[0].cpu().numpy() - ref["J"]).max() <= 1e-7
        assert np.abs(K[0].cpu().numpy() - ref["K"]).max() <= 1e-7
        assert abs(EJ[0] - ref["E_J"]) <= 1e-6 and abs(EK[0] - ref["E_K"]) <= 1e-6
        h.close()
    # a handle without the table keeps the defaults
    h = dfjk.Handle(I.molecule(6, seed=1006), precision=dfjk.DFJK_MIXED)
    assert h.tuning == [0, 0, 0, 0]
    h.close()
