"""Element-wise comparison of GPU factors with the oracle's, with tolerances
derived from each precision mode's rounding.

The tolerance of a factor X (L, U or B) is the oracle's own response to a
perturbation of the size that the mode's arithmetic introduces, times a
safety factor of 10:

  * the sketch: Y + eps_Y ||Y_i|| G_i / sqrt(l) for every row i (G standard
    normal), eps_Y = 4 u of the sketch's arithmetic (FP32 sums of the
    CountSketch buckets and a log2(l1)-stage FFT have a per-row relative
    error of a few u);
  * B = L_y^+ P A: B + eps_B (|W| |P A|) o G, eps_B = 4 u_32 for the FP32
    mode (B within FP32 parity), 2^-16 with W in two BF16 planes (the one-step
    refinement: W carries 16 bits) and 2^-8 with one plane;
  * L = L_y L_b: + sqrt(k) 4 u_32 (|L_y| |L_b|) o G (the FP32 product).

The oracle runs its own steps 3-7 (Algorithm 1) on the perturbed sketch, so
every input of these runs is the oracle's.  tau_X = 10 max over the draws of
max |X' - X| (relative to max |X| for L and B; U is bounded by 1).  Where the
perturbation moves the first k pivots of either LU, the factors are not
comparable entry by entry (the perturbed run picked other rows), and that
factor's tolerance is None.

L is compared in the original row order of A (row p[i] of the original
matrix holds row i of L), because rows of L past the first k pivot rows sit
in an order that steps k..l-1 of the panel LU choose among rounding-level
candidates for exactly low-rank inputs.
"""
import numpy as np
import scipy.sparse

import oracle

U32 = 2.0 ** -24
U64 = 2.0 ** -53
EPS_B = {"f64": 4 * U64, "f32": 4 * U32, "bf16_refine": 2.0 ** -16, "bf16": 2.0 ** -8}
SAFETY = 10.0


def _abs_product(W, PA):
    if scipy.sparse.issparse(PA):
        return np.asarray((abs(PA).T @ np.abs(W).T).T)
    return np.abs(W) @ np.abs(PA)


def _steps_3_to_7(A, Y, k, l, eps_B, eps_L, rng):
    """The oracle's steps 3-7 on a given sketch Y, with B and L perturbed."""
    ly = oracle.lu_partial_pivot(Y, steps=l)
    p = ly.perm
    Ly = oracle.unit_lower(ly.lu, k)
    W = oracle.pinv_householder(Ly)
    PA = oracle.rlu.row_gather(A, p)
    B = np.asarray((PA.T @ W.T).T) if scipy.sparse.issparse(PA) else W @ PA
    if eps_B:
        B = B + eps_B * _abs_product(W, PA) * rng.standard_normal(B.shape)
    lb = oracle.lu_partial_pivot(B.T, steps=k)
    q = lb.perm
    Lb = np.triu(lb.lu[:k, :k]).T
    Ub = oracle.unit_lower(lb.lu, k).T
    L = Ly @ Lb
    if eps_L:
        L = L + eps_L * (np.abs(Ly) @ np.abs(Lb)) * rng.standard_normal(L.shape)
    return L, Ub, B, p, q


def original_rows(L, p):
    out = np.empty_like(L)
    out[np.asarray(p)] = L
    return out


def tolerances(A, o, k, l, prec, draws=2, seed=0):
    """tau for L, U, B (None where the perturbation moves the pivots)."""
    eps_Y = 4 * (U64 if prec == "f64" else U32)
    eps_B = EPS_B[prec]
    eps_L = 0.0 if prec == "f64" else 4 * U32 * np.sqrt(k)
    rng = np.random.default_rng(seed)
    Lo = original_rows(o.L, o.p)
    worst = {"L": 0.0, "U": 0.0, "B": 0.0}
    moved_p = moved_q = False
    rn = np.linalg.norm(o.Y, axis=1, keepdims=True)
    for _ in range(draws):
        Yp = o.Y + eps_Y * rn * rng.standard_normal(o.Y.shape) / np.sqrt(o.Y.shape[1])
        L, U, B, p, q = _steps_3_to_7(A, Yp, k, l, eps_B, eps_L, rng)
        if not np.array_equal(p[:k], o.p[:k]):
            moved_p = True
            continue
        worst["B"] = max(worst["B"], np.abs(B - o.B).max() / np.abs(o.B).max())
        if not np.array_equal(q, o.q):
            moved_q = True
            continue
        worst["L"] = max(worst["L"], np.abs(original_rows(L, p) - Lo).max() / np.abs(Lo).max())
        worst["U"] = max(worst["U"], np.abs(U - o.U).max())
    tau = {x: SAFETY * v for x, v in worst.items()}
    if moved_p:
        tau = {"L": None, "U": None, "B": None}
    elif moved_q:
        tau["L"] = tau["U"] = None
    return tau


def check_elementwise(g, o, k, tau, B_gpu=None):
    """Compare the GPU's factors with the oracle's wherever the GPU picked the
    same pivots and the tolerance exists.  Returns the names compared and the
    relative differences found."""
    done = {}
    same_p = np.array_equal(g["p"][:k], o.p[:k])
    same_q = np.array_equal(g["q"], o.q)
    if same_p and B_gpu is not None and tau["B"] is not None:
        d = np.abs(B_gpu - o.B).max() / np.abs(o.B).max()
        assert d <= tau["B"], ("B", d, tau["B"])
        done["B"] = d
    if same_p and same_q and tau["L"] is not None:
        Lo = original_rows(o.L, o.p)
        d = np.abs(original_rows(g["L"], g["p"]) - Lo).max() / np.abs(Lo).max()
        assert d <= tau["L"], ("L", d, tau["L"])
        done["L"] = d
        d = np.abs(g["U"] - o.U).max()
        assert d <= tau["U"], ("U", d, tau["U"])
        done["U"] = d
    return done
