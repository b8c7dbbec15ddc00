"""Learned stage-time planner: choose between the uncut simulation and cutting
into n segments -- and the merge form and segment tile width of the cut --
from predicted stage times, with the closed-form thresholds of Eqs. 13-15 as
the fallback.

An ensemble of small fully connected networks (hand-written CUDA forward,
backward and Adam kernels behind ``cc_mlp_*``) maps circuit features to the
log10 of the four stage times (T_pre, T_sub, T_merge, T_orig of Eq. 3),
trained on times measured on this GPU.  Where the prediction error measured
on held-out instances near a query exceeds 20 % (the ensemble's spread where
no hold-out set is given), the planner answers with the closed-form
threshold instead.

Host logic and marshalling only; every network evaluation runs in the CUDA
kernels.
"""

from __future__ import annotations

import ctypes
import math
from ctypes import c_int32
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import capi

STAGES = ("pre", "sub", "merge", "orig")
FORMS = ("fma", "tf32x3", "f16x3", "bf16x3", "ozaki")
FEATURES = ("q", "log2_depth", "n", "cut_bits", "log2_n_sub", "max_seg_bits",
            "log2_dense_gates", "log2_two_qubit_gates", "seg_tile_bits") + tuple(
                "form_" + f for f in FORMS)
# max |dpsi| / max |psi| each merge form guarantees (cc_merge_form): the
# planner only picks a form whose bound meets the caller's tolerance
FORM_TOL = {"fma": 0.0, "tf32x3": 2e-6, "f16x3": 2e-6, "bf16x3": 5e-5, "ozaki": 1e-12}


def threshold(q: float, n: int) -> float:
    """Largest c_total for which T_sub < T_orig under the paper's cost model:
    Eq. 13 (n = 2: q/2) and Eq. 14 (n >= 3: q (n-1)^2 / (2n) +
    (n-1) log2(n / (n-2)) / 2)."""
    if n < 2:
        raise ValueError("a cut needs n >= 2")
    if n == 2:
        return q / 2.0
    return q * (n - 1) ** 2 / (2.0 * n) + (n - 1) * math.log2(n / (n - 2.0)) / 2.0


def nonuniform_threshold(q: float, n: int, dseg_over_d: float) -> float:
    """The threshold of Eqs. 13-14 lowered for segment depth D_seg (Eq. 15):
    T_sub < T_orig becomes N_sub 2^{-q (1 - 1/n)} D_seg / D < 1, which moves
    log2 N_sub by log2(n D_seg / D) against the uniform case D_seg = D / n,
    i.e. c_total by that times (n - 1) / 2 (n >= 3) or 1 (n = 2): 0 at
    D_seg = D / n, 1 cut (n = 2) and (n - 1) log2(n) / 2 cuts (n >= 3) at
    D_seg = D."""
    r = min(max(dseg_over_d, 1.0 / n), 1.0)
    shift = math.log2(n * r) * (1.0 if n == 2 else (n - 1) / 2.0)
    return threshold(q, n) - shift


def circuit_depth(gates, qubits=None) -> int:
    """Depth of the gate list (as-soon-as-possible layering); with `qubits`,
    of the gates that touch those qubits, a cut gate counting on both sides."""
    level = {}
    depth = 0
    for g in gates:
        qs = [g.q0] + ([g.q1] if g.q1 >= 0 else [])
        if qubits is not None:
            qs = [x for x in qs if x in qubits]
            if not qs:
                continue
        d = 1 + max(level.get(x, 0) for x in qs)
        for x in qs:
            level[x] = d
        depth = max(depth, d)
    return depth


def depth_ratio(gates, seg_sizes: Sequence[int]) -> float:
    """D_seg / D with D_seg the largest segment depth (contiguous segments)."""
    d = circuit_depth(gates)
    if d == 0:
        return 1.0 / len(seg_sizes)
    start, dseg = 0, 0
    for s in seg_sizes:
        dseg = max(dseg, circuit_depth(gates, set(range(start, start + s))))
        start += s
    return dseg / d


def features(q: int, depth: int, n: int, cut_bits: int, n_sub: int, max_seg_bits: int,
             dense_gates: int, two_qubit_gates: int, seg_tile_bits: int = 13,
             form: str = "fma") -> List[float]:
    return [float(q), math.log2(max(depth, 1)), float(n), float(cut_bits),
            math.log2(max(n_sub, 1)), float(max_seg_bits),
            math.log2(dense_gates + 1), math.log2(two_qubit_gates + 1),
            float(seg_tile_bits)] + [1.0 if form == f else 0.0 for f in FORMS]


class MLP:
    """One network: parameters, Adam state and workspace in device memory."""

    def __init__(self, dims: Sequence[int], seed: int, device="cuda"):
        self.dims = list(dims)
        self._dims_c = (c_int32 * len(self.dims))(*self.dims)
        n_p = capi.lib().cc_mlp_param_count(self._dims_c, len(self.dims) - 1)
        if n_p < 0:
            raise ValueError("bad layer widths")
        rng = np.random.default_rng(seed)
        flat = []
        for l in range(len(self.dims) - 1):  # He-uniform weights, zero biases
            lim = math.sqrt(6.0 / self.dims[l])
            flat.append(rng.uniform(-lim, lim, self.dims[l + 1] * self.dims[l]))
            flat.append(np.zeros(self.dims[l + 1]))
        self.params = torch.tensor(np.concatenate(flat), dtype=torch.float32, device=device)
        assert self.params.numel() == n_p
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self._work = None

    def _workspace(self, n: int) -> torch.Tensor:
        nb = capi.lib().cc_mlp_work_bytes(self._dims_c, len(self.dims) - 1, n)
        if self._work is None or self._work.numel() * 4 < nb:
            self._work = torch.empty((nb + 3) // 4, dtype=torch.float32, device=self.params.device)
        return self._work

    def train(self, x: torch.Tensor, t: torch.Tensor, epochs: int, lr: float) -> torch.Tensor:
        n = x.shape[0]
        work = self._workspace(n)
        loss = torch.empty(max(epochs, 1), dtype=torch.float32, device=x.device)
        capi.check(capi.lib().cc_mlp_train(
            self._dims_c, len(self.dims) - 1, self.params.data_ptr(), self.m.data_ptr(),
            self.v.data_ptr(), x.data_ptr(), t.data_ptr(), n, epochs, ctypes.c_float(lr),
            loss.data_ptr(), work.data_ptr(), work.numel() * 4,
            torch.cuda.current_stream().cuda_stream), "cc_mlp_train")
        return loss[:epochs]

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        n = x.shape[0]
        y = torch.empty((n, self.dims[-1]), dtype=torch.float32, device=x.device)
        work = self._workspace(n)
        capi.check(capi.lib().cc_mlp_forward(
            self._dims_c, len(self.dims) - 1, self.params.data_ptr(), x.data_ptr(), n,
            y.data_ptr(), work.data_ptr(), work.numel() * 4,
            torch.cuda.current_stream().cuda_stream), "cc_mlp_forward")
        return y


class StagePlanner:
    """Ensemble of MLPs predicting log10 stage seconds from circuit features
    (including the segment tile width and the merge form, so the planner
    picks those too).  Its fallback trigger is the prediction error measured
    on held-out instances near the query (set_holdout), or the ensemble's
    spread where no held-out error is known."""

    def __init__(self, n_models: int = 4, hidden: Sequence[int] = (64, 64, 64), seed: int = 0,
                 fallback_spread: float = 0.20, device="cuda"):
        self.hidden, self.seed, self.n_models = list(hidden), seed, n_models
        self.dims = None
        self.models = []  # built by fit() for the width of its features
        self.fallback_spread = fallback_spread
        self.fallback_error = fallback_spread
        self.device = device
        self.x_mu = self.x_sd = self.y_mu = self.y_sd = None
        self.hold_x = self.hold_err = None
        self.hold_k = 8

    def fit(self, X: np.ndarray, seconds: np.ndarray, epochs: int = 3000, lr: float = 2e-3):
        self.dims = [int(np.asarray(X).shape[1]), *self.hidden, len(STAGES)]
        self.models = [MLP(self.dims, self.seed + 1000 * i, self.device)
                       for i in range(self.n_models)]
        Y = np.log10(np.maximum(seconds, 1e-7))
        self.x_mu, self.x_sd = X.mean(0), X.std(0) + 1e-9
        self.y_mu, self.y_sd = Y.mean(0), Y.std(0) + 1e-9
        xt = torch.tensor((X - self.x_mu) / self.x_sd, dtype=torch.float32, device=self.device)
        yt = torch.tensor((Y - self.y_mu) / self.y_sd, dtype=torch.float32, device=self.device)
        return [m.train(xt, yt, epochs, lr).cpu().numpy() for m in self.models]

    def predict_members(self, X: np.ndarray) -> np.ndarray:
        """[n_models, n, 4] predicted seconds."""
        xt = torch.tensor((np.asarray(X, dtype=np.float64) - self.x_mu) / self.x_sd,
                          dtype=torch.float32, device=self.device)
        outs = [m.forward(xt).cpu().numpy().astype(np.float64) for m in self.models]
        return np.stack([10.0 ** (o * self.y_sd + self.y_mu) for o in outs])

    def predict(self, X: np.ndarray) -> Dict[str, np.ndarray]:
        """Ensemble mean of the stage seconds, T_cut, and the relative spread
        (std / mean across members) of T_cut and T_orig."""
        P = self.predict_members(X)
        t_cut = P[:, :, 0] + P[:, :, 1] + P[:, :, 2]
        t_orig = P[:, :, 3]
        out = {s: P[:, :, i].mean(0) for i, s in enumerate(STAGES)}
        out["cut"] = t_cut.mean(0)
        out["spread"] = np.maximum(t_cut.std(0) / t_cut.mean(0), t_orig.std(0) / t_orig.mean(0))
        return out

    def set_holdout(self, X: np.ndarray, seconds: np.ndarray):
        """Held-out instances and their measured stage seconds: the relative
        error of the predicted T_cut and T_orig on each becomes the error
        estimate of queries near it (the mean over its hold_k nearest
        neighbours in standardised feature space)."""
        pr = self.predict(X)
        t_cut = seconds[:, 0] + seconds[:, 1] + seconds[:, 2]
        e_cut = np.abs(pr["cut"] - t_cut) / t_cut
        e_orig = np.abs(pr["orig"] - seconds[:, 3]) / seconds[:, 3]
        self.hold_x = (np.asarray(X, dtype=np.float64) - self.x_mu) / self.x_sd
        self.hold_err = np.maximum(e_cut, e_orig)

    def expected_error(self, X: np.ndarray) -> Optional[np.ndarray]:
        """Held-out relative error near each query (None without a hold-out set)."""
        if self.hold_x is None:
            return None
        Z = (np.asarray(X, dtype=np.float64) - self.x_mu) / self.x_sd
        d = ((Z[:, None, :] - self.hold_x[None, :, :]) ** 2).sum(-1)
        k = min(self.hold_k, self.hold_x.shape[0])
        idx = np.argpartition(d, k - 1, axis=1)[:, :k]
        return self.hold_err[idx].mean(1)

    def decide(self, q: int, options: Sequence[dict], tol: float = 2e-6,
               dseg_over_d: Optional[float] = None) -> dict:
        """Choose among cutting options (dicts with 'n', 'form',
        'seg_tile_bits', 'features', 'cut_bits', 'n_sub') and the uncut
        simulation; only merge forms whose bound meets `tol` count.  Where the
        held-out error near any admissible option (or, without a hold-out set,
        the ensemble spread) exceeds the fallback level, the closed-form model
        decides instead: among the options whose c_total stays below Eqs.
        13-14 lowered by Eq. 15 for the circuit's D_seg / D, the one with the
        fewest cuts (then the fewest segments), else uncut; the merge form is
        then left to the library (AUTO).  Both the merge term k^{c_max} 2^q
        and the subcircuit count N_sub of Table I grow with the cuts, and
        measured chains of more segments with the same cuts per boundary
        merge far slower, so the fewest cuts is the safe pick when the model
        cannot be trusted."""
        opts = [o for o in options if FORM_TOL.get(o.get("form", "fma"), 0.0) <= tol]
        X = np.array([o["features"] for o in opts])
        pr = self.predict(X)
        err = self.expected_error(X)
        if err is not None:
            fallback = bool(np.any(err > self.fallback_error))
            reason = "held-out error"
        else:
            fallback = bool(np.any(pr["spread"] > self.fallback_spread))
            reason = "ensemble spread"
        ratio = 1.0 if dseg_over_d is None else dseg_over_d
        out = {"pred_cut": pr["cut"].tolist(), "pred_orig": float(pr["orig"].mean()),
               "spread": pr["spread"].tolist(),
               "expected_error": None if err is None else err.tolist()}
        if fallback:
            ok = [o for o in opts if o["cut_bits"] < nonuniform_threshold(q, o["n"], ratio)]
            if ok:
                best = min(ok, key=lambda o: (o["cut_bits"], o["n"]))
                out.update(choice=best["n"], form="auto", seg_tile_bits=None)
            else:
                out.update(choice=0, form=None, seg_tile_bits=None)
            out.update(fallback=True, reason=reason)
            return out
        best = int(np.argmin(pr["cut"]))
        t_orig = float(pr["orig"].mean())
        if pr["cut"][best] < t_orig:
            o = opts[best]
            out.update(choice=o["n"], form=o.get("form"), seg_tile_bits=o.get("seg_tile_bits"))
        else:
            out.update(choice=0, form=None, seg_tile_bits=None)
        out.update(fallback=False, reason=None)
        return out


def max_feasible_q(predict_seconds, budget_s: float, q_max: int, q_min: int = 1) -> Optional[int]:
    """Largest q in q_min..q_max whose predicted seconds fit the budget
    (predictions increase with q); None if even q_min does not."""
    best = None
    for q in range(q_min, q_max + 1):
        if predict_seconds(q) <= budget_s:
            best = q
    return best
