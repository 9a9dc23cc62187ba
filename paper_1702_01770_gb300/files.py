"""Host-side file helpers around the boundary: AB sequences in and the per-iteration
multicanonical data out (Sec. 3.2, SET_PROT-SEQ and the output files of the
MUCA engine; Sec. 3.3).  No device work and none of the method's arithmetic
beyond restating the weights as the coefficients of Eq. 8."""
import numpy as np


def read_sequences(path) -> list:
    """AB sequences, one chain per line (A or B letters, any case; blanks and
    text after '#' ignored).  Returns one uint8 array per chain (0 = A, 1 = B),
    the layout phast_system.seq takes when concatenated."""
    chains = []
    with open(path) as fh:
        for no, line in enumerate(fh, 1):
            text = "".join(line.split("#", 1)[0].split()).upper()
            if not text:
                continue
            bad = set(text) - {"A", "B"}
            if bad:
                raise ValueError(f"{path}:{no}: letters other than A and B: {''.join(sorted(bad))}")
            chains.append(np.frombuffer(text.encode(), dtype=np.uint8).copy() - ord("A"))
    if not chains:
        raise ValueError(f"{path}: no sequence")
    return chains


def muca_coefficients(lnW, e_min: float, bin_width: float):
    """The coefficients of Eq. 8 behind a tabulated log-weight: ln W(E) = -beta_k E
    + alpha_k on [E_k, E_{k+1}] through the bin centres E_k = e_min + (k + 1/2) w,
    so beta_k = (lnW_k - lnW_{k+1}) / w and alpha_k = lnW_k + beta_k E_k,
    k = 0 .. K-2 (S_muca(E_k) = beta_k E_k - alpha_k = -lnW_k)."""
    lnW = np.asarray(lnW, dtype=np.float64)
    Ek = e_min + (np.arange(lnW.size - 1) + 0.5) * bin_width
    beta = (lnW[:-1] - lnW[1:]) / bin_width
    alpha = lnW[:-1] + beta * Ek
    return beta, alpha


def save_iteration(path, iteration: int, lnW, e_min: float, bin_width: float, hist=None, g_acc=None):
    """One multicanonical iteration as a .npz file: lnW, the coefficients beta and
    alpha of Eq. 8, the histogram (summed over walkers, or per jackknife block) and
    the Berg recursion's accumulated weights g, whichever are given (tensors or
    arrays; device tensors are copied to the host)."""
    def host(x):
        if x is None:
            return None
        if hasattr(x, "detach"):
            x = x.detach().cpu().numpy()
        return np.asarray(x)

    lnW = host(lnW)
    beta, alpha = muca_coefficients(lnW, e_min, bin_width)
    out = {"iteration": np.int64(iteration), "e_min": np.float64(e_min), "bin_width": np.float64(bin_width),
           "lnW": lnW, "beta": beta, "alpha": alpha}
    if hist is not None:
        out["hist"] = host(hist)
    if g_acc is not None:
        out["g_acc"] = host(g_acc)
    np.savez(path, **out)
