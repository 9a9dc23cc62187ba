"""Host-side file helpers: sequence reader and the per-iteration output."""
import numpy as np
import pytest

from paper_1702_01770_gb300 import files, inputs


def test_read_sequences(tmp_path):
    p = tmp_path / "seqs.txt"
    p.write_text("# two chains\nABBAB ABBAB\n\n  bab  # trailing comment\n")
    s = files.read_sequences(p)
    assert [x.tolist() for x in s] == [[0, 1, 1, 0, 1, 0, 1, 1, 0, 1], [1, 0, 1]]
    assert np.array_equal(s[0], inputs.str_to_seq("ABBABABBAB"))
    p.write_text("ABX\n")
    with pytest.raises(ValueError, match="X"):
        files.read_sequences(p)


def test_coefficients_restate_the_weights():
    rng = np.random.default_rng(3)
    lnW = np.cumsum(rng.standard_normal(50))
    e_min, w = -3.0, 0.2
    beta, alpha = files.muca_coefficients(lnW, e_min, w)
    Ek = e_min + (np.arange(49) + 0.5) * w
    assert np.allclose(-beta * Ek + alpha, lnW[:-1], rtol=0, atol=1e-12)          # at E_k
    assert np.allclose(-beta * (Ek + w) + alpha, lnW[1:], rtol=0, atol=1e-12)     # at E_{k+1}


def test_save_iteration(tmp_path):
    lnW = -0.1 * np.arange(20.0)
    files.save_iteration(tmp_path / "it7.npz", 7, lnW, 0.0, 0.5, hist=np.arange(20), g_acc=np.ones(19))
    d = np.load(tmp_path / "it7.npz")
    assert int(d["iteration"]) == 7 and np.allclose(d["beta"], 0.2) and d["alpha"].size == 19
    assert np.array_equal(d["hist"], np.arange(20)) and np.array_equal(d["lnW"], lnW)
