"""Ghost-track classifier: training on the GPU through the C ABI.

The network (10 -> 32 -> 32 -> 1, BF16 forward, FP32 accumulation and master
weights, Adam) scores fitted track candidates; with ``Params.use_mlp = 1`` a
reconstruction keeps the candidates whose logit reaches
``Params.mlp_logit_threshold`` instead of applying the plain cuts.  Every
computation runs in the library's kernels (``velo_mlp_*``); this module only
moves arrays and loops over epochs.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np

from . import velo as _v

N_PARAMS = 1441
N_IN = 10


def init_params(seed: int) -> np.ndarray:
    """He-style initialisation from a seeded generator (float32, 1441)."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0, math.sqrt(2.0 / N_IN), (32, N_IN))
    w2 = rng.normal(0, math.sqrt(2.0 / 32), (32, 32))
    w3 = rng.normal(0, math.sqrt(1.0 / 32), 32)
    return np.concatenate([w1.ravel(), np.zeros(32), w2.ravel(), np.zeros(32), w3, [0.0]]).astype(np.float32)


def standardisation(features: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per-feature mean and inverse standard deviation (float32)."""
    f = np.asarray(features, np.float64)
    mean = f.mean(0)
    std = f.std(0)
    return mean.astype(np.float32), (1.0 / np.where(std > 1e-12, std, 1.0)).astype(np.float32)


@dataclasses.dataclass
class TrainState:
    params: np.ndarray       # float32 master weights
    params_bf16: np.ndarray  # uint16 BF16 copy used by the forward pass
    m1: np.ndarray
    m2: np.ndarray
    step: int
    mean: np.ndarray
    istd: np.ndarray

    def save(self, path: str):
        np.savez(path, params=self.params, params_bf16=self.params_bf16, m1=self.m1, m2=self.m2,
                 step=self.step, mean=self.mean, istd=self.istd)

    @staticmethod
    def load(path: str) -> "TrainState":
        z = np.load(path)
        return TrainState(z["params"], z["params_bf16"], z["m1"], z["m2"], int(z["step"]), z["mean"], z["istd"])


class Trainer:
    """Owns a velo_mlp_trainer; features and labels live on the device."""

    def __init__(self, params: np.ndarray, mean: np.ndarray, istd: np.ndarray, max_batch: int = 1024):
        self.lib = _v.load_library()
        self.mean = np.ascontiguousarray(mean, np.float32)
        self.istd = np.ascontiguousarray(istd, np.float32)
        p = np.ascontiguousarray(params, np.float32)
        self.max_batch = max_batch
        self.t = ctypes.c_void_p()
        _v._check(self.lib.velo_mlp_create(p.ctypes.data, self.mean.ctypes.data, self.istd.ctypes.data, max_batch,
                                           ctypes.byref(self.t)), "velo_mlp_create")

    def close(self):
        if self.t:
            self.lib.velo_mlp_destroy(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, feats, labels, lr: float, stream: int = 0):
        """One Adam step on device tensors feats [n, 10] float32, labels [n] float32."""
        n = int(labels.numel())
        _v._check(self.lib.velo_mlp_step(self.t, feats.data_ptr(), labels.data_ptr(), n, ctypes.c_float(lr),
                                         ctypes.c_void_p(stream)), "velo_mlp_step")

    def gradient(self, feats, labels, stream: int = 0) -> tuple[np.ndarray, float]:
        g = np.zeros(N_PARAMS, np.float32)
        loss = ctypes.c_float()
        n = int(labels.numel())
        _v._check(self.lib.velo_mlp_gradient(self.t, feats.data_ptr(), labels.data_ptr(), n, g.ctypes.data,
                                             ctypes.byref(loss), ctypes.c_void_p(stream)), "velo_mlp_gradient")
        return g, float(loss.value)

    def logits(self, feats, stream: int = 0):
        import torch
        n = int(feats.shape[0])
        out = torch.empty(max(n, 1), dtype=torch.float32, device=feats.device)
        _v._check(self.lib.velo_mlp_logits(self.t, feats.data_ptr(), n, out.data_ptr(), ctypes.c_void_p(stream)),
                  "velo_mlp_logits")
        return out[:n]

    def state(self) -> TrainState:
        p = np.zeros(N_PARAMS, np.float32)
        pb = np.zeros(N_PARAMS, np.uint16)
        m1 = np.zeros(N_PARAMS, np.float32)
        m2 = np.zeros(N_PARAMS, np.float32)
        st = ctypes.c_uint32()
        _v._check(self.lib.velo_mlp_get_state(self.t, p.ctypes.data, pb.ctypes.data, m1.ctypes.data, m2.ctypes.data,
                                              ctypes.byref(st)), "velo_mlp_get_state")
        return TrainState(p, pb, m1, m2, int(st.value), self.mean.copy(), self.istd.copy())

    def restore(self, s: TrainState):
        _v._check(self.lib.velo_mlp_set_state(self.t, np.ascontiguousarray(s.params, np.float32).ctypes.data,
                                              np.ascontiguousarray(s.m1, np.float32).ctypes.data,
                                              np.ascontiguousarray(s.m2, np.float32).ctypes.data, s.step),
                  "velo_mlp_set_state")


def train(features: np.ndarray, labels: np.ndarray, epochs: int = 20, batch: int = 1024, lr: float = 1e-3,
          seed: int = 3, device: str = "cuda", trainer: Trainer | None = None, start_epoch: int = 0) -> Trainer:
    """Trains on (features [n, 10] float32, labels [n]) with shuffled batches
    (a seeded permutation per epoch); returns the trainer."""
    import torch
    f = torch.from_numpy(np.ascontiguousarray(features, np.float32)).to(device)
    y = torch.from_numpy(np.ascontiguousarray(labels, np.float32)).to(device)
    if trainer is None:
        mean, istd = standardisation(features)
        trainer = Trainer(init_params(seed), mean, istd, batch)
    n = len(labels)
    for ep in range(start_epoch, epochs):
        perm = torch.from_numpy(np.random.default_rng(seed * 1000 + ep).permutation(n)).to(device)
        fs, ys = f[perm].contiguous(), y[perm].contiguous()
        for b0 in range(0, n - batch + 1, batch):
            trainer.step(fs[b0:b0 + batch], ys[b0:b0 + batch], lr)
    torch.cuda.synchronize()
    return trainer


def logit_threshold_for_efficiency(logits: np.ndarray, labels: np.ndarray, keep_fraction_of_real: float) -> float:
    """Largest logit threshold that keeps at least the given fraction of the
    real (label 1) candidates."""
    real = np.sort(np.asarray(logits, np.float32)[np.asarray(labels) > 0.5])
    if len(real) == 0:
        return 0.0
    k = int(math.floor((1.0 - keep_fraction_of_real) * len(real)))
    return float(real[min(max(k, 0), len(real) - 1)])
