"""One small, fixed invocation of a hot-path kernel, for profiler captures.

Usage:
    python -m paper_1902_10559_gb300.profile_case realistic [--iters N] [--kernel K] [--lpc L] [--threads T]
    python -m paper_1902_10559_gb300.profile_case batch --slices S [--iters N] [--kernel K] [--dtype f32|bf16|f16] ...
    python -m paper_1902_10559_gb300.profile_case multi [--nrhs R] [--iters N] [--rc C] [--dtype f32|bf16|f16]
    python -m paper_1902_10559_gb300.profile_case cnn [--batch B]

Each case builds its inputs, runs the kernel twice, and exits. The first run is
a warm-up: skip it with ncu's `-s 1`. The launch shape is given on the command
line, not tuned, so a capture is the same from run to run.
"""
from __future__ import annotations

import argparse
import ctypes


def main():
    import torch

    from . import splitsart as ss
    from .synthetic import REALISTIC, TINY, batch_geometries, cnn_initial_params, random_phantom

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["realistic", "batch", "multi", "cnn"])
    ap.add_argument("--slices", type=int, default=16)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--lpc", type=int, default=4)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0, help="kernels 7 and 8: chunk entry target (0 = library default)")
    ap.add_argument("--lpr", type=int, default=0, help="lanes per row (kernels 7 and 8; multi); 0 = library default")
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--rc", type=int, default=0, help="multi: right-hand sides per CTA (0 = library choice)")
    ap.add_argument("--dtype", choices=["f32", "bf16", "f16"], default="f32",
                    help="multi and batch: matrix value storage")
    args = ap.parse_args()
    dev = torch.device("cuda")

    def phantoms(gs, config_id, n_ell):
        import numpy as np
        imgs = [random_phantom(g, config_id, n_ell, stream=2 * k) for k, g in enumerate(gs)]
        return torch.as_tensor(np.concatenate([im.reshape(-1) for im in imgs]), dtype=torch.float32, device=dev)

    if args.case in ("realistic", "batch"):
        if args.case == "realistic":
            gs = [REALISTIC]
            sysm = ss.fold_system(ss.make_geometry(REALISTIC), ss.F32)
        else:
            gs = batch_geometries()[: args.slices]
            sysm = ss.fold_batch([ss.make_geometry(g) for g in gs], ss.DTYPE_NAMES[args.dtype])
        p = torch.empty(sysm.M, device=dev)
        ss.project(sysm, phantoms(gs, 2 if args.case == "realistic" else 3, 12), p, layout=ss.LAYOUT_IMAGE)
        p12 = torch.empty(sysm.Mh, 2, device=dev)
        ss.fold_rhs(sysm, p, p12)
        f12 = torch.zeros(sysm.Nh, 2, device=dev)
        opts = ss.solve_opts(args.iters, 0.8, kernel=args.kernel, lanes_per_col=args.lpc, tile_entries=args.tile,
                             lanes_per_row=args.lpr,
                             block_threads=args.threads)
        for _ in range(2):
            f12.zero_()
            ss.solve(sysm, p12, f12, opts)
        torch.cuda.synchronize()
        print("S", sysm.info()["S"], "result", ss.solve_result(sysm))
    elif args.case == "multi":
        sysm = ss.fold_system(ss.make_geometry(TINY), ss.DTYPE_NAMES[args.dtype])
        vec = ss.fold_batch([ss.make_geometry(TINY)] * args.nrhs, ss.F32)
        p = torch.empty(vec.M, device=dev)
        ss.project(vec, phantoms([TINY] * args.nrhs, 3, 8), p, layout=ss.LAYOUT_IMAGE)
        p12 = torch.empty(args.nrhs, TINY.M // 2, 2, device=dev)
        ss.fold_rhs(vec, p, p12.view(-1, 2))
        f12 = torch.zeros(args.nrhs, TINY.N // 2, 2, device=dev)
        info = torch.zeros(args.nrhs * ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device=dev)
        for _ in range(2):
            f12.zero_()
            ss.solve_multi(sysm, p12, f12, ss.solve_opts(args.iters, 0.8, block_threads=args.threads,
                                                          lanes_per_row=args.lpr), info, rhs_per_cta=args.rc)
        torch.cuda.synchronize()
        print("multi", ss.read_infos(info, 1)[0])
    else:
        net = ss.Cnn(TINY.nz, TINY.nx, args.batch, cnn_initial_params())
        net.set_mode(1)
        x = torch.rand(args.batch, TINY.nz, TINY.nx, device=dev)
        t = torch.rand_like(x)
        y = torch.empty_like(x)
        loss = torch.zeros(1, device=dev)
        for _ in range(2):
            net.forward(x, y)
            net.train_step(x, t, lr=1e-3, loss=loss)
        torch.cuda.synchronize()
        print("cnn loss", float(loss.item()))


if __name__ == "__main__":
    main()
