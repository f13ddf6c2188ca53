"""Learned warm start for split-SART: data, training, and the comparison with plain SART.

Steps, all run by the library's kernels through the C ABI:
1. Training data: each seeded phantom (tiny-slice geometry) is projected,
   solved for 5 and 500 iterations from zero, and recombined as images
   [nz][nx]. The 5-iteration image is the network input and the
   500-iteration image the target.
2. Training: the network (splitsart_cnn_*) with Adam on mini-batches.
3. Warm-started solve, for each right-hand side:
   - run 5 iterations;
   - apply the network to the recombined image;
   - fold the network's image into (f1, f2) (proof of Theorem 1);
   - keep it only if its residual is lower than a zero start's (rho < 1);
     otherwise fall back to plain split-SART, continuing from the
     5-iteration image;
   - continue split-SART until rho <= tol.
   Measured on held-out phantoms, a guess can raise rho above the 5-iteration
   image's and still reach the tolerance in fewer iterations. So the fallback
   guards against a useless network (no better than zero), not against that.
4. The comparison is plain split-SART from zero, to the same tolerance.

Many right-hand sides are processed at once with splitsart_solve_multi. The
vector folds use a batch of copies of the slice, which has exactly the
[nrhs][M] / [nrhs][Mh] layouts.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import splitsart as ss
from .synthetic import TINY, cnn_initial_params, random_phantom

EARLY_ITERS = 5
TARGET_ITERS = 500


class WarmStart:
    def __init__(self, g=TINY, chunk: int = 1024, max_batch: int = 256, params=None, mode: int = 1,
                 lam: float = 1.0, rhs_per_cta: int = 1):
        import torch
        self.g = g
        self.lam = lam
        # One right-hand side per CTA: with more right-hand sides than resident slots,
        # the persistent multi-RHS launch refills each slot as its right-hand side
        # stops, so the time follows the mean iteration count, not the slowest one.
        self.rhs_per_cta = rhs_per_cta
        self.geom = ss.make_geometry(g)
        self.system = ss.fold_system(self.geom, ss.F32)
        self.chunk = chunk
        # [n][...] layouts for the vector folds: a batch of n copies of the slice, made once per n.
        self._vecs = {chunk: ss.fold_batch([self.geom] * chunk, ss.F32)}
        self.cnn = ss.Cnn(g.nz, g.nx, max_batch, cnn_initial_params() if params is None else params)
        self.steps = 0  # Adam steps taken
        if mode:
            self.cnn.set_mode(mode)
        self.dev = torch.device("cuda")

    # ---- helpers over chunks of right-hand sides ----
    def _chunks(self, n):
        for a in range(0, n, self.chunk):
            yield a, min(a + self.chunk, n)

    def _vec_for(self, n):
        if n not in self._vecs:
            self._vecs[n] = ss.fold_batch([self.geom] * n, ss.F32)
        return self._vecs[n]

    def project(self, images):
        """images: CUDA float32 [n][nz][nx] -> p [n][M]."""
        import torch
        g = self.g
        n = images.shape[0]
        p = torch.empty(n, g.M, device=self.dev)
        for a, b in self._chunks(n):
            v = self._vec_for(b - a)
            ss.project(v, images[a:b].reshape(-1), p[a:b].reshape(-1), layout=ss.LAYOUT_IMAGE)
        return p

    def fold_rhs(self, p):
        import torch
        n = p.shape[0]
        p12 = torch.empty(n, self.g.M // 2, 2, device=self.dev)
        for a, b in self._chunks(n):
            ss.fold_rhs(self._vec_for(b - a), p[a:b].reshape(-1), p12[a:b].reshape(-1, 2))
        return p12

    def recombine(self, f12):
        import torch
        n = f12.shape[0]
        img = torch.empty(n, self.g.nz, self.g.nx, device=self.dev)
        for a, b in self._chunks(n):
            ss.recombine(self._vec_for(b - a), f12[a:b].reshape(-1, 2), img[a:b].reshape(-1), layout=ss.LAYOUT_IMAGE)
        return img

    def fold_image(self, img):
        import torch
        n = img.shape[0]
        f12 = torch.empty(n, self.g.N // 2, 2, device=self.dev)
        for a, b in self._chunks(n):
            ss.fold_image(self._vec_for(b - a), img[a:b].reshape(-1), f12[a:b].reshape(-1, 2), layout=ss.LAYOUT_IMAGE)
        return f12

    def solve(self, p12, f12, iters, tol=0.0, order=None):
        """Solve all right-hand sides in place (in queue `order` if given); returns the raw device info."""
        import torch
        n = p12.shape[0]
        info = torch.zeros(n * ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device=self.dev)
        ss.solve_multi(self.system, p12, f12, ss.solve_opts(iters, self.lam, tol), info, rhs_per_cta=self.rhs_per_cta,
                       order=order)
        return info

    # ---- 1. data ----
    def phantoms(self, seeds):
        import torch
        imgs = np.stack([random_phantom(self.g, 5, 8, stream=int(s)) for s in seeds]).astype(np.float32)
        return torch.as_tensor(imgs, device=self.dev)

    def make_pairs(self, seeds):
        """Return (x, t): 5-iteration and 500-iteration images [n][nz][nx] of the seeded phantoms."""
        import torch
        truth = self.phantoms(seeds)
        p12 = self.fold_rhs(self.project(truth))
        f12 = torch.zeros(len(seeds), self.g.N // 2, 2, device=self.dev)
        self.solve(p12, f12, EARLY_ITERS)
        x = self.recombine(f12)
        self.solve(p12, f12, TARGET_ITERS - EARLY_ITERS)
        t = self.recombine(f12)
        return x, t

    # ---- 2. training ----
    def train(self, x, t, epochs=10, batch=64, lr=1e-3, seed=0, log_every=0, checkpoint=None):
        """Adam on mini-batches. With ``checkpoint`` (a path), the weights, the
        Adam moments and the step count are written there after every epoch."""
        import torch
        n = x.shape[0]
        rng = np.random.default_rng(seed)
        loss = torch.zeros(1, device=self.dev)
        hist = []
        for ep in range(epochs):
            order = torch.as_tensor(rng.permutation(n), device=self.dev)
            acc = torch.zeros(1, device=self.dev, dtype=torch.float64)
            steps = 0
            for a in range(0, n - batch + 1, batch):
                idx = order[a:a + batch]
                xb, tb = x[idx].contiguous(), t[idx].contiguous()
                self.cnn.train_step(xb, tb, lr=lr, loss=loss)
                acc += loss.double()
                steps += 1
            self.steps += steps
            hist.append(float(acc.item() / max(steps, 1)))
            if checkpoint:
                self.save(checkpoint, epoch=ep + 1, loss=hist[-1])
            if log_every and (ep + 1) % log_every == 0:
                print(f"epoch {ep + 1}: mean loss {hist[-1]:.4e}", flush=True)
        return hist

    def save(self, path, **meta):
        """Write the network's weights, Adam moments and step count to ``path`` (.npz)."""
        p, m, v = self.cnn.params(moments=True)
        np.savez(path, params=p, m=m, v=v, step=np.int64(self.steps), **{k: np.asarray(x) for k, x in meta.items()})

    def load(self, path):
        """Resume from a file written by ``save``: training continues exactly where it stopped."""
        z = np.load(path)
        self.steps = int(z["step"])
        self.cnn.set_params(z["params"], z["m"], z["v"], step=self.steps)

    def predict(self, x):
        import torch
        y = torch.empty_like(x)
        for a in range(0, x.shape[0], self.cnn.max_batch):
            b = min(a + self.cnn.max_batch, x.shape[0])
            self.cnn.forward(x[a:b].contiguous(), y[a:b])
        return y

    # ---- 3./4. warm-started and plain solves to rho <= tol ----
    def solve_plain(self, p12, tol, max_iters):
        """Plain split-SART from zero. Returns (f12, info)."""
        import torch
        f = torch.zeros(p12.shape[0], self.g.N // 2, 2, device=self.dev)
        return f, self.solve(p12, f, max_iters, tol)

    def solve_warm(self, p12, tol, max_iters, longest_first=True):
        """5 iterations, network, fold, fallback, continue. Returns (f12, info_early, info_rest, picked).

        A right-hand side that met tol within the first 5 iterations has
        stopped there; the continuation then returns it unchanged with 0
        further iterations. With longest_first, the continuation's persistent
        launch takes the right-hand sides in decreasing order of their start's
        rho (the guess's where it was kept, else the 5-iteration image's), so
        the slowest ones start first and the launch's tail is shorter.
        """
        import torch
        n = p12.shape[0]
        f_warm = torch.zeros(n, self.g.N // 2, 2, device=self.dev)
        info_early = self.solve(p12, f_warm, EARLY_ITERS, tol)
        guess = self.fold_image(self.predict(self.recombine(f_warm)))
        info_guess = self.solve(p12, guess, 0)  # rho of the guess
        info_zero = self.solve(p12, torch.zeros_like(guess), 0)  # rho of a zero start (1, or 0 if p = 0)
        picked = torch.zeros(n, dtype=torch.int32, device=self.dev)
        ss.pick_start(self.system, guess, info_guess, info_zero, f_warm, picked)
        order = None
        if longest_first:
            rho_guess = np.array([i["rho"] for i in ss.read_infos(info_guess, n)])
            rho_early = np.array([i["rho"] for i in ss.read_infos(info_early, n)])
            rho_start = np.where(picked.cpu().numpy() != 0, rho_guess, rho_early)
            order = torch.as_tensor(np.argsort(-rho_start, kind="stable").astype(np.int32), device=self.dev)
        info_rest = self.solve(p12, f_warm, max_iters - EARLY_ITERS, tol, order=order)
        self._last_guess_info = info_guess
        return f_warm, info_early, info_rest, picked

    @staticmethod
    def warm_counts(early, rest, tol):
        """Per right-hand side: total iterations and final rho of the warm-started solve."""
        its = np.array([e["iters"] if e["rho"] <= tol else EARLY_ITERS + r["iters"] for e, r in zip(early, rest)])
        rho = np.array([e["rho"] if e["rho"] <= tol else r["rho"] for e, r in zip(early, rest)])
        return its, rho

    def compare(self, seeds, tol=1e-3, max_iters=20000):
        """Plain split-SART from zero vs the warm start, on the seeded phantoms.

        Returns per-RHS iteration counts, timings, and the fraction of warm starts kept.
        """
        import torch
        truth = self.phantoms(seeds)
        p12 = self.fold_rhs(self.project(truth))
        n = len(seeds)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record()
        _, info_plain = self.solve_plain(p12, tol, max_iters)
        ev[1].record()
        ev[2].record()
        _, info_early, info_rest, picked = self.solve_warm(p12, tol, max_iters)
        ev[3].record()
        torch.cuda.synchronize()
        plain = ss.read_infos(info_plain, n)
        early = ss.read_infos(info_early, n)
        rest = ss.read_infos(info_rest, n)
        it_warm, rho_warm = self.warm_counts(early, rest, tol)
        return {
            "n": n, "tol": tol,
            "iters_plain": np.array([i["iters"] for i in plain]), "iters_warm": it_warm,
            "rho_plain": np.array([i["rho"] for i in plain]), "rho_warm": rho_warm,
            "ms_plain": ev[0].elapsed_time(ev[1]), "ms_warm": ev[2].elapsed_time(ev[3]),
            "warm_kept": float(picked.float().mean().item()),
            "rho_early": np.array([e["rho"] for e in early]),
            "rho_guess": np.array([i["rho"] for i in ss.read_infos(self._last_guess_info, n)]),
        }
