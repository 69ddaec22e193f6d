"""Parameter choice for a DKSS product: the thesis's rule, measurement, and a
learned cost model that decides which candidates are worth measuring.

The search space is dkss_plan_candidates(N) (include/dkss.h): every valid
(M, m, u, p, z) the library has kernels for.  Candidates that run the same
kernels on the same shapes (equal M, m, u, L, LR, levels, last-level length)
cost the same whatever p is, so only one of each is kept.

* rule_choice: Section 4.1 of the thesis picks p^z just above the coefficient
  bound, the largest u that fits, then the smallest M m, keeping M/m near
  N / log^3 N.  No measurement.
* measure: device time of one product (CUDA events, median of repeats).
* CostModel: the network of dkss_mlp_* (features -> predicted log2 ms),
  trained on the GPU with the library's own forward, gradient and Adam
  kernels.  choose() measures only the model's top-k candidates.
"""
import json
import math

import numpy as np

from . import binding

FEATURES = 12          # DKSS_MLP_FEATURES
HIDDEN = 32            # DKSS_MLP_HIDDEN
NPARAM = 1505          # DKSS_MLP_PARAMS
KEY = ("M", "m", "u", "L", "LR", "levels", "r_last")


def candidates(n_bits):
    """Valid parameter sets for N-bit operands, one per distinct kernel shape."""
    seen, out = set(), []
    for c in binding.plan_candidates(n_bits):
        k = tuple(c[f] for f in KEY)
        if k not in seen:
            seen.add(k)
            out.append(c)
    return out


def features(n_bits, c):
    """12 scaled features of a candidate (inputs of the cost model)."""
    lg = math.log2
    rmuls = (3 * (c["levels"] - 1) + 1) * c["P2"]
    work = rmuls * c["m"] * lg(c["m"]) * c["LR"] ** 2
    nbytes = c["P2"] * c["m"] * c["L"] * 4 * (2 * c["levels"] + 1)
    return np.array([lg(n_bits) / 32, lg(c["M"]) / 24, lg(c["m"]) / 6, c["u"] / 32, c["L"] / 4, c["LR"] / 5,
                     c["levels"] / 4, lg(c["r_last"]) / 7, lg(c["P2"]) / 24, lg(rmuls) / 30, lg(work) / 40,
                     lg(nbytes) / 40], dtype=np.float32)


def rule_choice(n_bits, cands):
    """The thesis's rule (Section 4.1): largest u, then smallest M m, then M/m
    closest to N / log2(N)^3, then the fewest limbs."""
    target = n_bits / math.log2(n_bits) ** 3
    return min(cands, key=lambda c: (-c["u"], c["M"] * c["m"], abs(math.log2(c["M"] / c["m"]) - math.log2(target)),
                                     c["L"], c["LR"], c["z"]))


def timing_operands(n_bits, device="cuda", seed=0):
    """Random N-bit operands on the device (their values do not change the time)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    words = (n_bits + 63) // 64
    a = torch.randint(-(1 << 63), (1 << 63) - 1, (words,), generator=g, dtype=torch.int64)
    b = torch.randint(-(1 << 63), (1 << 63) - 1, (words,), generator=g, dtype=torch.int64)
    top = n_bits - 64 * (words - 1)
    if top < 64:
        mask = (1 << top) - 1
        a[-1] = int(a[-1]) & mask
        b[-1] = int(b[-1]) & mask
    return a.to(device), b.to(device)


def measure(n_bits, c, reps=5, warmup=2, operands=None):
    """Median device time (ms) of one product with candidate c."""
    import torch
    a, b = operands if operands is not None else timing_operands(n_bits)
    with binding.Plan(n_bits, c["M"], c["m"], c["u"], c["p"], c["z"]) as plan:
        out = torch.empty(2 * a.numel(), dtype=torch.int64, device=a.device)
        for _ in range(warmup):
            plan.mul(a, b, out)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.mul(a, b, out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


class CostModel:
    """Predicts log2(ms) of a product from its 12 features.  Weights live on the
    device; training and prediction run the library's dkss_mlp_* kernels."""

    def __init__(self, seed=0, device="cuda"):
        import torch
        rng = np.random.default_rng(seed)
        parts = [rng.normal(0, math.sqrt(2.0 / FEATURES), HIDDEN * FEATURES), np.zeros(HIDDEN),
                 rng.normal(0, math.sqrt(2.0 / HIDDEN), HIDDEN * HIDDEN), np.zeros(HIDDEN),
                 rng.normal(0, math.sqrt(1.0 / HIDDEN), HIDDEN), np.zeros(1)]
        p = np.concatenate(parts).astype(np.float32)
        assert p.size == NPARAM
        self.device = device
        self.params = torch.from_numpy(p).to(device)
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        self.y_shift = 0.0

    def _x(self, x):
        import torch
        return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32)).to(self.device).contiguous()

    def predict(self, x):
        """Predicted log2(ms) for rows of features (numpy, float32)."""
        import torch
        xd = self._x(x)
        y = torch.empty(xd.shape[0], dtype=torch.float32, device=self.device)
        lib = binding.load()
        binding._check(lib.dkss_mlp_forward(self.params.data_ptr(), xd.data_ptr(), xd.shape[0], y.data_ptr(),
                                            binding._stream_handle(None)), "dkss_mlp_forward")
        return y.cpu().numpy().astype(np.float64) + self.y_shift

    def gradient(self, x, t):
        """(loss, gradient) of the mean squared error on (x, t) with the current weights."""
        xd = self._x(x)
        td = self._x(t)
        lib = binding.load()
        binding._check(lib.dkss_mlp_grad(self.params.data_ptr(), xd.data_ptr(), td.data_ptr(), xd.shape[0],
                                         self.grad.data_ptr(), self.loss.data_ptr(), binding._stream_handle(None)),
                       "dkss_mlp_grad")
        return float(self.loss.item()), self.grad.cpu().numpy()

    def fit(self, x, t, steps=3000, lr=3e-3):
        """Full-batch Adam on log2(ms) targets; returns the loss history."""
        t = np.asarray(t, dtype=np.float64)
        self.y_shift = float(t.mean())
        xd = self._x(x)
        td = self._x(t - self.y_shift)
        lib = binding.load()
        st = binding._stream_handle(None)
        hist = []
        for _ in range(steps):
            binding._check(lib.dkss_mlp_grad(self.params.data_ptr(), xd.data_ptr(), td.data_ptr(), xd.shape[0],
                                             self.grad.data_ptr(), self.loss.data_ptr(), st), "dkss_mlp_grad")
            self.step += 1
            binding._check(lib.dkss_mlp_adam(self.params.data_ptr(), self.grad.data_ptr(), self.m1.data_ptr(),
                                             self.m2.data_ptr(), lr, self.step, st), "dkss_mlp_adam")
            if self.step % 100 == 0:
                hist.append(float(self.loss.item()))
        return hist

    def save(self, path):
        with open(path, "w") as f:
            json.dump({"params": self.params.cpu().numpy().tolist(), "y_shift": self.y_shift}, f)

    @classmethod
    def load(cls, path, device="cuda"):
        import torch
        with open(path) as f:
            d = json.load(f)
        m = cls(device=device)
        m.params = torch.tensor(d["params"], dtype=torch.float32, device=device)
        m.y_shift = d["y_shift"]
        return m


def collect(n_list, reps=5):
    """Measured (features, log2 ms, candidate, ms) for every candidate of each N."""
    rows = []
    for n in n_list:
        ops = timing_operands(n)
        for c in candidates(n):
            ms = measure(n, c, reps=reps, operands=ops)
            rows.append((features(n, c), math.log2(ms), c, ms, n))
    return rows


def choose(n_bits, model, trials=3, operands=None):
    """Measure the model's `trials` best-predicted candidates; return
    (candidate, ms, trials used)."""
    cands = candidates(n_bits)
    pred = model.predict(np.stack([features(n_bits, c) for c in cands]))
    order = np.argsort(pred)[:max(1, trials)]
    ops = operands if operands is not None else timing_operands(n_bits)
    timed = [(measure(n_bits, cands[i], operands=ops), cands[i]) for i in order]
    ms, best = min(timed, key=lambda x: x[0])
    return best, ms, len(order)
