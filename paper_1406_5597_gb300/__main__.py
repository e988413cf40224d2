"""One-shot driver: a plan, one forward r2c and one inverse c2r on seeded
random data on the current CUDA device, through the C ABI.

    python -m paper_1406_5597_gb300 --shape 512,512,512 [--flags 0x40] [--dtype f32|bf16x3|f16|f64]
    python -m paper_1406_5597_gb300 --shape 256,256,256 --ns
    python -m paper_1406_5597_gb300 --shape 256,256,256 --nl
    python -m paper_1406_5597_gb300 --shape 64,1024,2048 --forms 1,6

Prints the plan description and the round-trip relative L2 error
(c2r(r2c(x)) / N against x).  With --ns it instead runs one pseudo-spectral
Navier-Stokes step (fft3d_ns_step, direct launches) on random spectra, with
--nl two applications of the nonlinear term (fft3d_nonlinear_exec, direct
launches: a warm-up and the one a profiler skips to).  Useful
as the target of a profiler run: it launches exactly the kernels of one
transform pair (or one step).
"""
import argparse

import torch

from . import FFT3D_F32, FFT3D_F32_TC_BF16X3, FFT3D_F32_TC_F16, FFT3D_F64, NavierStokes, NonlinearTerm, Plan, load


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--shape", default="512,512,512", help="n0,n1,n2")
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--flags", type=lambda v: int(v, 0), default=0, help="FFT3D_FLAG_* bits")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16x3", "f16", "f64"])
    ap.add_argument("--seed", type=int, default=1408)
    ap.add_argument("--ns", action="store_true", help="one Navier-Stokes step instead of r2c + c2r")
    ap.add_argument("--nl", action="store_true", help="nonlinear-term applications instead of r2c + c2r")
    ap.add_argument("--forms", default=None, help="column forms f0,f1 of the n0 and n1 passes (fft3d_set_choices)")
    args = ap.parse_args()
    n0, n1, n2 = (int(v) for v in args.shape.split(","))
    dtype = {"f32": FFT3D_F32, "bf16x3": FFT3D_F32_TC_BF16X3, "f16": FFT3D_F32_TC_F16, "f64": FFT3D_F64}[args.dtype]
    rt, ct = (torch.float64, torch.complex128) if dtype == FFT3D_F64 else (torch.float32, torch.complex64)
    load()
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(args.seed)
    if args.ns:
        ns = NavierStokes(n0, n1, n2)
        u = torch.randn((3, n0, n1, n2 // 2 + 1), dtype=torch.complex64, device=dev, generator=gen)
        ns.step(u, 0.01, 1e-3, stream=False)
        torch.cuda.synchronize(dev)
        print(f"one Navier-Stokes step at {n0}x{n1}x{n2}: |u| = {float(u.abs().norm()):.6e}")
        ns.close()
        return
    if args.nl:
        nl = NonlinearTerm(n0, n1, n2)
        u = torch.randn((3, n0, n1, n2 // 2 + 1), dtype=torch.complex64, device=dev, generator=gen)
        out = torch.empty((6, n0, n1, n2 // 2 + 1), dtype=torch.complex64, device=dev)
        for _ in range(2):
            nl(u, out=out, stream=False)
        torch.cuda.synchronize(dev)
        print(f"nonlinear term at {n0}x{n1}x{n2}: |N| = {float(out.abs().norm()):.6e}")
        nl.close()
        return
    lead = (args.batch,) if args.batch > 1 else ()
    x = torch.randn(lead + (n0, n1, n2), device=dev, generator=gen, dtype=rt)
    X = torch.empty(lead + (n0, n1, n2 // 2 + 1), dtype=ct, device=dev)
    y = torch.empty_like(x)
    plan = Plan(n0, n1, n2, dtype, args.batch, args.flags)
    if args.forms:
        from . import fft3d_get_choices, fft3d_set_choices
        ch = fft3d_get_choices(plan.handle)
        ch[3], ch[4] = (int(v) for v in args.forms.split(","))
        if fft3d_set_choices(plan.handle, ch) != 0:
            raise SystemExit(f"forms {args.forms}: not available for this plan")
    s = torch.cuda.current_stream(dev).cuda_stream
    plan.r2c(x.data_ptr(), X.data_ptr(), s)
    plan.c2r(X.data_ptr(), y.data_ptr(), s)
    torch.cuda.synchronize(dev)
    err = float((y / (n0 * n1 * n2) - x).norm() / x.norm())
    print(f"{plan.describe()}; round trip rel-L2 {err:.3e}")
    plan.close()


if __name__ == "__main__":
    main()
