"""Learned stage-time planner: choose between the uncut simulation and cutting
into n segments from predicted stage times, with the closed-form thresholds
of Eqs. 13-14 as the fallback.

An ensemble of small fully connected networks (hand-written CUDA forward,
backward and Adam kernels behind ``cc_mlp_*``) maps circuit features to the
log10 of the four stage times (T_pre, T_sub, T_merge, T_orig of Eq. 3),
trained on times measured on this GPU.  The ensemble's spread stands in for
the prediction error: where it exceeds ``fallback_spread`` (20 %) the
planner answers with the closed-form threshold instead.

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
FEATURES = ("q", "log2_depth", "n", "cut_bits", "log2_n_sub", "max_seg_bits",
            "log2_dense_gates", "log2_two_qubit_gates")


def threshold(q: float, n: int) -> float:
    """Largest c_total for which T_sub < T_orig under the paper's cost model:
    Eq. 13 (n = 2: q/2) and Eq. 14 (n >= 3: q (n-1)^2 / (2n) +
    (n-1) log2(n / (n-2)) / 2)."""
    if n < 2:
        raise ValueError("a cut needs n >= 2")
    if n == 2:
        return q / 2.0
    return q * (n - 1) ** 2 / (2.0 * n) + (n - 1) * math.log2(n / (n - 2.0)) / 2.0


def features(q: int, depth: int, n: int, cut_bits: int, n_sub: int, max_seg_bits: int,
             dense_gates: int, two_qubit_gates: int) -> List[float]:
    return [float(q), math.log2(max(depth, 1)), float(n), float(cut_bits),
            math.log2(max(n_sub, 1)), float(max_seg_bits),
            math.log2(dense_gates + 1), math.log2(two_qubit_gates + 1)]


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
    """Ensemble of MLPs predicting log10 stage seconds from circuit features."""

    def __init__(self, n_models: int = 4, hidden: Sequence[int] = (64, 64, 64), seed: int = 0,
                 fallback_spread: float = 0.20, device="cuda"):
        self.dims = [len(FEATURES), *hidden, len(STAGES)]
        self.models = [MLP(self.dims, seed + 1000 * i, device) for i in range(n_models)]
        self.fallback_spread = fallback_spread
        self.device = device
        self.x_mu = self.x_sd = self.y_mu = self.y_sd = None

    def fit(self, X: np.ndarray, seconds: np.ndarray, epochs: int = 3000, lr: float = 2e-3):
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

    def decide(self, q: int, options: Sequence[dict]) -> dict:
        """Choose among cutting options (dicts with 'n', 'features',
        'cut_bits', 'n_sub') and the uncut simulation.  Where the ensemble
        spread of any option exceeds the fallback level, the closed-form model
        decides instead: among the options whose c_total stays below Eq. 13/14,
        the one with the least subcircuit work N_sub 2^{q/n} / n (Table I),
        else uncut."""
        X = np.array([o["features"] for o in options])
        pr = self.predict(X)
        if np.any(pr["spread"] > self.fallback_spread):
            ok = [o for o in options if o["cut_bits"] < threshold(q, o["n"])]
            choice = min(ok, key=lambda o: o["n_sub"] * 2.0 ** (q / o["n"]) / o["n"])["n"] \
                if ok else 0
            return {"choice": choice, "fallback": True, "pred_cut": pr["cut"].tolist(),
                    "pred_orig": float(pr["orig"].mean()), "spread": pr["spread"].tolist()}
        best = int(np.argmin(pr["cut"]))
        t_orig = float(pr["orig"].mean())
        choice = options[best]["n"] if pr["cut"][best] < t_orig else 0
        return {"choice": choice, "fallback": False, "pred_cut": pr["cut"].tolist(),
                "pred_orig": t_orig, "spread": pr["spread"].tolist()}


def max_feasible_q(predict_seconds, budget_s: float, q_max: int, q_min: int = 1) -> Optional[int]:
    """Largest q in q_min..q_max whose predicted seconds fit the budget
    (predictions increase with q); None if even q_min does not."""
    best = None
    for q in range(q_min, q_max + 1):
        if predict_seconds(q) <= budget_s:
            best = q
    return best
