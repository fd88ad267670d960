"""Run one libotm operator (or design steps) on seeded inputs, for timing and
for profiling a single kernel under ncu.

  python opbench.py --op apply_K --n 128 --reps 3
  python opbench.py --op step --n 128 --reps 2 --warmup 3

Ops: apply_K, gs (one fine colour pass), filter, kappa_sens, oc, step,
unet (network forward), unet_train (one Adam step), conv3 (one convolution,
--cin/--cout).
Prints the mean CUDA-event time per repetition.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="apply_K")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--dtype", type=int, default=1, help="1 = FP32, 0 = FP64; precision for --op step (2 = mixed)")
    ap.add_argument("--colour", type=int, default=8, help="--op gs: colour (0-7) or group pass 8 + g")
    ap.add_argument("--widths", default="16,32,64,128", help="--op unet*: network widths")
    ap.add_argument("--smoother", type=int, default=0, help="--op step: coarse_smoother (0 GS, 1 Chebyshev)")
    ap.add_argument("--optimizer", type=int, default=0, help="--op step: 0 OC (model 3), 1 MMA (model 2)")
    ap.add_argument("--cin", type=int, default=16)
    ap.add_argument("--cout", type=int, default=16)
    ap.add_argument("--async", dest="async_", action="store_true",
                    help="--op apply_K: queue the stream-ordered entry point back to back (no host sync per call)")
    args = ap.parse_args()

    import torch
    from paper_2405_19991_gb300 import otm
    import workloads as W

    n, N = args.n, args.n ** 3
    dev = "cuda:0"
    t = torch.float64 if args.dtype == 0 else torch.float32
    st = torch.cuda.current_stream()
    rng = np.random.default_rng(0)
    rho = torch.as_tensor(W.initial_density(n, 0.3, 1), dtype=t, device=dev)
    k = (1e-3 + rho ** 3 * (1 - 1e-3)).contiguous()
    u = torch.as_tensor(rng.standard_normal(3 * N), dtype=t, device=dev)
    out = torch.empty(3 * N, dtype=t, device=dev)
    s = torch.as_tensor(-np.abs(rng.standard_normal(N)), dtype=t, device=dev)
    ctx = None
    unet = None
    if args.op.startswith("unet"):
        widths = [int(v) for v in args.widths.split(",")]
        unet = otm.otm_unet_create(n, widths, 0, st.cuda_stream)
        y = torch.empty(3 * N, dtype=torch.float32, device=dev)
        tgt = torch.as_tensor(rng.standard_normal(3 * N), dtype=torch.float32, device=dev)
        rho32 = rho.float().contiguous()
    if args.op == "conv3":
        xin = torch.randn((N, args.cin), device=dev).to(torch.bfloat16)
        wc = (torch.randn((27, args.cin, args.cout), device=dev) / (27 * args.cin) ** 0.5).to(torch.bfloat16)
        bc = torch.zeros(args.cout, device=dev)
        yc = torch.empty((N, args.cout), dtype=torch.bfloat16, device=dev)
    ctx_bytes = 0
    if args.op == "step":
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        p = otm.otm_params_default(n=n, precision=args.dtype, kappa_target=W.TARGET_ORTHOTROPIC, rmin=2.0,
                                   stream=st.cuda_stream, coarse_smoother=args.smoother,
                                   optimizer=args.optimizer)
        ctx = otm.otm_create_ex(p)
        r0 = W.initial_density(n, 0.3, 1).astype(np.float32)
        otm.otm_set_density(ctx, r0.ctypes.data, 0)
        torch.cuda.synchronize()
        ctx_bytes = free0 - torch.cuda.mem_get_info()[0]

    def run():
        if args.op == "apply_K" and args.async_:
            otm.otm_op_apply_K_async(args.dtype, n, k, u, out, st.cuda_stream)
        elif args.op == "apply_K":
            otm.otm_op_apply_K(args.dtype, n, k, u, out, st.cuda_stream)
        elif args.op == "gs":
            otm.otm_op_gs_colour(args.dtype, n, k, u, out, args.colour, st.cuda_stream)
        elif args.op == "filter":
            otm.otm_op_filter_simp(args.dtype, n, 2.0, 3.0, 1.0, 1e-3, rho, out, out[N:], st.cuda_stream)
        elif args.op == "kappa_sens":
            otm.otm_op_kappa_sens(args.dtype, n, 3.0, 1.0, 1e-3, k, rho, u, [1, 1, 1, 0, 0, 0], out,
                                  st.cuda_stream)
        elif args.op == "oc":
            otm.otm_op_oc_update(args.dtype, n, 0.29, 0.05, 0.5, 1e-3, rho, s, out, st.cuda_stream)
        elif args.op == "step":
            otm.otm_step(ctx)
        elif args.op == "unet":
            otm.otm_unet_forward(unet, rho32, y, st.cuda_stream)
        elif args.op == "unet_train":
            otm.otm_unet_train_step(unet, rho32, tgt, 1e-4, 1.0, st.cuda_stream)
        elif args.op == "conv3":
            otm.otm_op_conv3(n, args.cin, args.cout, xin, wc, bc, 1, yc, st.cuda_stream)
        else:
            raise SystemExit(f"unknown op {args.op}")

    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.reps):
        run()
    e1.record(st)
    torch.cuda.synchronize()
    print(f"{args.op} n={n}: {e0.elapsed_time(e1) / args.reps * 1e3:.1f} us per repetition")
    if args.op == "step":
        info, _ = otm.otm_step(ctx)
        print(f"  PCG iterations per load case {list(info.cg_iters)}, resid {max(info.resid):.2e}")
        print(f"  tensor + sensitivity + design update {info.stage_ms[4] * 1e3:.1f} us, g {info.g:.3e}, "
              f"multiplier {info.lambda_:.3e}, context device memory {ctx_bytes / 2**20:.1f} MiB")
    if args.op == "conv3":
        flops = 2.0 * N * 27 * args.cin * args.cout
        print(f"conv3 {args.cin}->{args.cout}: {flops / (e0.elapsed_time(e1) / args.reps * 1e-3) / 1e12:.1f} TFLOP/s")
    if ctx is not None:
        otm.otm_destroy(ctx)
    if unet is not None:
        otm.otm_unet_destroy(unet)


if __name__ == "__main__":
    main()
