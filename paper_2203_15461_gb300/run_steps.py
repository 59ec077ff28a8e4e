"""Run the graph-captured charge update of the EDL capacitor (4,320 sites, 8 replicas of 5,700
charges) for a fixed number of steps and exit: a plain driver for an external profiler, which
times nothing itself.  One step is one replay of cpm_step_graph (electrolyte vector b, S product,
neutrality), the same step bench.py times.  With --s-product-only the driver instead runs the
single-precision S product (cpm_update on a random b) of the 16,384-site two-sheet graphene
capacitor that bench.py measures against the HBM peak.

    python -m paper_2203_15461_gb300.run_steps --steps 4 [--k-prec f16x2|fp32] [--replicas 8]
    python -m paper_2203_15461_gb300.run_steps --steps 4 --s-product-only
    python -m paper_2203_15461_gb300.run_steps --steps 4 --tc-product --sites 8192 --replicas 256
    python -m paper_2203_15461_gb300.run_steps --steps 4 --p3m 32,32,128,7

With --tc-product the driver runs the batched tensor-core S product (S as three bf16 planes,
persistent tcgen05 kernel with its tuned tile plan) of a two-sheet graphene capacitor of --sites
sites (8,192 or 16,384) on a random b of --replicas replicas.  With --p3m Kx,Ky,Kz,order the EDL step
takes the reciprocal part of b from P3M on that mesh instead of the Ewald sum.
"""
import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--k-prec", default="f16x2", choices=["fp32", "f16x2"])
    ap.add_argument("--s-product-only", action="store_true")
    ap.add_argument("--tc-product", action="store_true")
    ap.add_argument("--sites", type=int, default=8192, choices=[8192, 16384])
    ap.add_argument("--plan", default="", help="BN,stages,splits,ctas of the tensor-core product (default: tuned)")
    ap.add_argument("--p3m", default="", help="Kx,Ky,Kz,order: P3M reciprocal part of b (default: Ewald)")
    args = ap.parse_args()

    import torch

    from . import systems as s
    from .cpm import CPM

    if args.tc_product:
        cells = (32, 16) if args.sites == 8192 else (32, 32)
        el = s.graphene_plates(cells[0], cells[1], 2, 40.0, alpha=0.1, rcut=35.0)
        m = args.replicas
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = CPM.for_electrodes(el, s_prec="bf16x3", k_prec="fp32", stream=st).setup(el)
            ctx.cpm_release_assembly()
            if args.plan:
                ctx.cpm_gemm_set_plan(m, *[int(v) for v in args.plan.split(",")])
            plan = ctx.cpm_gemm_plan(m)
            b = torch.as_tensor(np.random.default_rng(7).normal(0.0, 1.0, (m, el.n)), device="cuda")
            psi = torch.as_tensor(np.tile([0.0, 1.0], (m, 1)), device="cuda")
            q = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
            qt = torch.empty((m,), dtype=torch.float64, device="cuda")
            for _ in range(args.steps):
                ctx.cpm_update(m, psi, b, q, qt)
        st.synchronize()
        print(f"{args.steps} tensor-core S products, n = {el.n}, m = {m}, plan {plan}, "
              f"max |sum q| = {float(qt.abs().max()):.3e}")
        return

    if args.s_product_only:
        el = s.graphene_plates(32, 32, 2, 40.0, alpha=0.1, rcut=35.0)
        m = args.replicas
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = CPM.for_electrodes(el, s_prec="fp32", k_prec="fp32", stream=st).setup(el)
            b = torch.as_tensor(np.random.default_rng(7).normal(0.0, 1.0, (m, el.n)), device="cuda")
            psi = torch.as_tensor(np.tile([0.0, 1.0], (m, 1)), device="cuda")
            q = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
            qt = torch.empty((m,), dtype=torch.float64, device="cuda")
            for _ in range(args.steps):
                ctx.cpm_update(m, psi, b, q, qt)
        st.synchronize()
        print(f"{args.steps} S products, n = {el.n}, max |sum q| = {float(qt.abs().max()):.3e}")
        return

    el, _, psi = s.workload_edl_capacitor(seed=1)
    m = args.replicas
    reps = [s.workload_edl_capacitor(seed=100 + r)[1] for r in range(m)]
    ne = max(e.n for e in reps)
    xyz = np.zeros((m, ne, 3))
    Q = np.zeros((m, ne))
    for r, e in enumerate(reps):
        xyz[r, :e.n] = e.xyz
        Q[r, :e.n] = e.Q
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        kw = {}
        if args.p3m:
            v = [int(t) for t in args.p3m.split(",")]
            kw["p3m"] = (tuple(v[:3]), v[3])
        ctx = CPM.for_electrodes(el, s_prec="fp32", k_prec=args.k_prec, stream=st, **kw).setup(el)
        dx = torch.as_tensor(xyz.reshape(-1, 3), device="cuda")
        dQ = torch.as_tensor(Q.reshape(-1), device="cuda")
        dp = torch.as_tensor(np.tile(psi, (m, 1)), device="cuda")
        b = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
        q = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
        qt = torch.empty((m,), dtype=torch.float64, device="cuda")
        for _ in range(args.steps):
            ctx.cpm_step_graph(m, ne, dx, dQ, dp, b, q, qt)
    st.synchronize()
    print(f"{args.steps} steps, max |sum q| = {float(qt.abs().max()):.3e}")


if __name__ == "__main__":
    main()
