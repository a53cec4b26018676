"""Per-workload report: iterations, true residual and the phi and E error of
the GPU solves against the FP64 oracle, for the five workloads of the solve.

Test infrastructure: it imports the oracle, which only the tests, the smoke
check and the benchmark's CPU leg may use.  Two commands:

  python tests/report_configs.py oracle512 [--out PATH]
      The oracle's FP64 solve of the 512^3 two-channel workload (a CPU job of
      about an hour and some 35 GB of host memory).  Stores its iteration
      count, true residual, and phi and E at seeded sample cells (plus three
      lines through the channels and heads) in
      tests/golden/twochannel512_oracle_samples.npz.

  python tests/report_configs.py gpu [--json PATH]
      On a GPU: the constant-coefficient 32^3 and channel 128^3 problems in
      FP64, the channel 256^3 problem at contrast 1e1, 1e3, 1e4 in mixed and
      FP64 precision, the 512^3 two-channel problem in mixed precision with an
      FP32 field, and the adjoint checks at 32^3 and 64^3.  The oracle solves
      the first five cases meanwhile in spawned processes; phi and E are
      compared in every cell (the 512^3 case at the stored sample cells).
      Errors are the largest element difference over the largest |oracle|.
      Prints a markdown table.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SAMPLES_512 = os.path.join(ROOT, "tests", "golden", "twochannel512_oracle_samples.npz")
SAMPLE_SEED = 4242
N_RANDOM_SAMPLES = 4096


def sample_cells(n: int) -> np.ndarray:
    """Linear indices of the 512^3 comparison: seeded random cells and three
    lines along z through the channel axes and the domain centre."""
    rng = np.random.default_rng(SAMPLE_SEED)
    idx = rng.choice(n ** 3, size=N_RANDOM_SAMPLES, replace=False)
    lines = []
    for cx, cy in ((0.4, 0.5), (0.6, 0.5), (0.5, 0.5)):
        i, j = int(cx * n), int(cy * n)
        lines.append(np.arange(n) * n * n + j * n + i)
    return np.unique(np.concatenate([idx] + lines))


def _oracle_case(args):
    """One oracle solve: phi, E (FP64) and the solve's iterations."""
    name, workload, n, kappa = args
    from oracle import gmg_oracle as O
    from streamer_inputs import make_inputs
    inp = make_inputs(workload, n=n, kappa=kappa)
    t0 = time.time()
    p = O.OracleParams()
    phi, info, _ = O.solve(p, inp["a"], inp["f"])
    grid = O.Grid(n, n, n)
    e = O.field_from_potential(grid, phi, p.phi_bottom, p.phi_top)
    return name, {"phi": phi, "e": np.stack(e), "iterations": info.iterations,
                  "true_rel_residual": info.true_rel_residual, "seconds": time.time() - t0}


def cmd_oracle512(out: str) -> None:
    name, r = _oracle_case(("twochannel512", "twochannel512", 512, None))
    n = 512
    idx = sample_cells(n)
    np.savez_compressed(out, cells=idx, phi=r["phi"].ravel()[idx], ex=r["e"][0].ravel()[idx],
                        ey=r["e"][1].ravel()[idx], ez=r["e"][2].ravel()[idx], iterations=r["iterations"],
                        true_rel_residual=r["true_rel_residual"], seconds=r["seconds"])
    print(f"oracle 512^3: {r['iterations']} iterations, true residual {r['true_rel_residual']:.3e}, "
          f"{r['seconds']:.0f} s; {idx.size} sample cells -> {out}")


def _maxrel(x, ref):
    return float(np.abs(np.asarray(x) - np.asarray(ref)).max() / np.abs(ref).max())


def cmd_gpu(json_out: str | None) -> None:
    cases = [("config 1: const 32^3", "const32", 32, None), ("config 2: channel 128^3", "channel128", 128, None)]
    for k in (1e1, 1e3, 1e4):
        cases.append((f"config 3: channel 256^3, kappa {k:g}", "channel256", 256, k))
    ctx_mp = mp.get_context("spawn")
    pool = ctx_mp.Pool(len(cases))
    pending = pool.map_async(_oracle_case, cases)

    import torch
    from oracle import gmg_oracle as O
    from paper_1812_08606_gb300 import build, gmg
    from streamer_inputs import make_inputs
    build.build()
    gmg.load()
    dev = torch.device("cuda:0")

    def gpu_solve(workload, n, kappa, prec, field_fp32=False):
        inp = make_inputs(workload, n=n, kappa=kappa)
        p = gmg.gmg_default_params(n, n, n, precision=prec)
        a = torch.from_numpy(inp["a"]).to(dev)
        f = torch.from_numpy(inp["f"]).to(dev)
        ctx = gmg.gmg_setup(p, a)
        phi = torch.zeros_like(f)
        torch.cuda.synchronize()
        t0 = time.time()
        gmg.gmg_update_coefficient(ctx, a)
        info = gmg.fgmres_solve(ctx, f, phi)
        torch.cuda.synchronize()
        ms = (time.time() - t0) * 1e3
        dt = torch.float32 if field_fp32 else torch.float64
        e = [torch.empty_like(f, dtype=dt) for _ in range(3)]
        gmg.field_from_potential(ctx, phi, *e)
        torch.cuda.synchronize()
        ctx.close()
        return inp, phi, torch.stack(e).double(), info, ms

    gpu = {}
    for name, wl, n, k in cases:
        precs = [gmg.GMG_PREC_FP64] if not name.startswith("config 3") else [gmg.GMG_PREC_MIXED, gmg.GMG_PREC_FP64]
        for prec in precs:
            inp, phi, e, info, ms = gpu_solve(wl, n, k, prec)
            gpu[(name, prec)] = (phi.cpu().numpy(), e.cpu().numpy(), info, ms, inp)
    rows = []
    oracle = dict(pending.get())
    pool.close()
    for (name, prec), (phi, e, info, ms, inp) in gpu.items():
        r = oracle[name]
        n = phi.shape[0]
        grid = O.Grid(n, n, n)
        b = O.assemble_rhs(grid, inp["a"], inp["f"], 0.0, 1.0)
        tr = float(np.linalg.norm(b - O.apply_operator(grid, inp["a"], phi)) / np.linalg.norm(b))
        rows.append({"case": name, "precision": "FP64" if prec == gmg.GMG_PREC_FP64 else "mixed",
                     "iterations": info.iterations, "oracle_iterations": r["iterations"],
                     "true_rel_residual": tr, "phi_err": _maxrel(phi, r["phi"]), "e_err": _maxrel(e, r["e"]),
                     "setup_solve_ms": round(ms, 2), "oracle_s": round(r["seconds"], 1)})
    # config 4 at the stored sample cells
    if os.path.exists(SAMPLES_512):
        s = np.load(SAMPLES_512)
        inp, phi, e, info, ms = gpu_solve("twochannel512", 512, None, gmg.GMG_PREC_MIXED, field_fp32=True)
        cells = torch.from_numpy(s["cells"]).to(dev)
        ph = phi.reshape(-1)[cells].cpu().numpy()
        es = e.reshape(3, -1)[:, cells].cpu().numpy()
        ref_e = np.stack([s["ex"], s["ey"], s["ez"]])
        rows.append({"case": "config 4: two channels 512^3 (sample cells)", "precision": "mixed, E FP32",
                     "iterations": info.iterations, "oracle_iterations": int(s["iterations"]),
                     "true_rel_residual": info.true_rel_residual, "phi_err": _maxrel(ph, s["phi"]),
                     "e_err": _maxrel(es, ref_e), "setup_solve_ms": round(ms, 2),
                     "oracle_s": round(float(s["seconds"]), 1), "samples": int(s["cells"].size)})
        del phi, e
    rows.append(adjoint_rows(torch, gmg, O, dev))
    print("| case | precision | iterations (oracle) | true residual | max phi error | max E error | set-up + solve ms |")
    print("|---|---|---|---|---|---|---|")
    for r in rows[:-1]:
        print(f"| {r['case']} | {r['precision']} | {r['iterations']} ({r['oracle_iterations']}) | "
              f"{r['true_rel_residual']:.2e} | {r['phi_err']:.2e} | {r['e_err']:.2e} | {r['setup_solve_ms']} |")
    print(json.dumps(rows[-1]))
    if json_out:
        with open(json_out, "w") as fh:
            json.dump(rows, fh, indent=1, default=float)


def adjoint_rows(torch, gmg, O, dev):
    """Config 5: central differences at 32^3 (64 seeded entries of a and f,
    steps 1e-6 and 1e-3 relative for a; at 1e-6 also with each solve's
    first-order error lambda . r~ added, r~ = b - A x~ from the oracle's
    operator, lambda from its adjoint solve) and the CPU adjoint at 64^3."""
    from paper_1812_08606_gb300 import PoissonSolver
    from streamer_inputs import make_inputs
    out = {"case": "config 5: adjoint"}
    inp = make_inputs("adjoint", n=32)
    shape = inp["a"].shape
    solver = PoissonSolver(shape, rtol=1e-13, precision=gmg.GMG_PREC_MIXED, max_iters=60)
    a = torch.from_numpy(inp["a"]).to(dev).requires_grad_(True)
    f = torch.from_numpy(inp["f"]).to(dev).requires_grad_(True)
    w = torch.from_numpy(inp["w"]).to(dev)
    (w * solver.solve(a, f)).sum().backward()
    ga, gf = a.grad.cpu().numpy(), f.grad.cpu().numpy()
    idx = np.random.default_rng(20181225).choice(a.numel(), size=64, replace=False)
    base_a, base_f = a.detach().clone(), f.detach().clone()
    prm = solver.params
    grid = O.Grid(shape[2], shape[1], shape[0], prm.lx, prm.ly, prm.lz)
    op = O.OracleParams(lx=prm.lx, ly=prm.ly, lz=prm.lz, phi_bottom=prm.phi_bottom, phi_top=prm.phi_top,
                        rtol=1e-13, max_iters=60)
    lam_o, _, _ = O.solve(op, inp["a"], inp["w"], homogeneous=True)

    def L(av, fv):
        with torch.no_grad():
            phi = solver.solve(av, fv)
            val = float((w * phi).sum())
        an, fn, ph = (t.cpu().numpy() for t in (av, fv, phi))
        r = O.assemble_rhs(grid, an, fn, prm.phi_bottom, prm.phi_top) - O.apply_operator(grid, an, ph)
        return val, float(np.sum(lam_o * r))
    for which, step in (("a", 1e-6), ("a", 1e-3), ("f", None)):
        errs, errs_c = [], []
        for q in idx:
            grad, base = (ga, base_a) if which == "a" else (gf, base_f)
            v = abs(float(base.view(-1)[q]))
            h = step * v if which == "a" else max(v, 1.0)
            plus, minus = base.clone(), base.clone()
            plus.view(-1)[q] += h
            minus.view(-1)[q] -= h
            (lp, ep), (lm, em) = (L(plus, base_f), L(minus, base_f)) if which == "a" else (L(base_a, plus), L(base_a, minus))
            sc = lambda x: max(abs(x), 1e-4 * np.abs(grad).max())
            fd, fdc = (lp - lm) / (2 * h), ((lp + ep) - (lm + em)) / (2 * h)
            errs.append(abs(grad.ravel()[q] - fd) / sc(fd))
            errs_c.append(abs(grad.ravel()[q] - fdc) / sc(fdc))
        out[f"fd_{which}_{step}"] = {"median": float(np.median(errs)), "max": float(np.max(errs))}
        if which == "a" and step == 1e-6:
            out[f"fd_{which}_{step}_corrected"] = {"median": float(np.median(errs_c)), "max": float(np.max(errs_c))}
    inp = make_inputs("adjoint", n=64)
    shape = inp["a"].shape
    solver = PoissonSolver(shape, rtol=1e-12)
    a = torch.from_numpy(inp["a"]).to(dev).requires_grad_(True)
    f = torch.from_numpy(inp["f"]).to(dev).requires_grad_(True)
    (torch.from_numpy(inp["w"]).to(dev) * solver.solve(a, f)).sum().backward()
    op = O.OracleParams(rtol=1e-12)
    phi, _, hier = O.solve(op, inp["a"], inp["f"])
    lam, _, _ = O.solve(op, inp["a"], inp["w"], homogeneous=True, hierarchy=hier)
    ga_ref = O.adjoint_coefficient_grad(O.Grid(64, 64, 64), phi, lam, 0.0, 1.0)
    out["cpu_adjoint_64"] = {"dLdf_max_err": _maxrel(f.grad.cpu().numpy(), lam),
                             "dLda_max_err": _maxrel(a.grad.cpu().numpy(), ga_ref)}
    return out


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    o = sub.add_parser("oracle512")
    o.add_argument("--out", default=SAMPLES_512)
    g = sub.add_parser("gpu")
    g.add_argument("--json", default=None)
    args = ap.parse_args()
    if args.cmd == "oracle512":
        cmd_oracle512(args.out)
    else:
        cmd_gpu(args.json)


if __name__ == "__main__":
    main()
