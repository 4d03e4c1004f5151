"""Write the stored expected values under tests/golden/ from the FP64 oracle only.

Usage:  python tests/golden/make_golden.py [name ...]

For each named workload (``microstructures.config_inputs``) this runs the
oracle's projected CG (O1) on the full grid to a relative residual of
``TOL`` and stores the effective tangent (mean-stress form, Mandel) with the
iteration counts.  ``disc32`` is also solved by the assembled FEM (O2) and
both results are stored.  ``lognormal64`` additionally stores the oracle's
adjoint gradient of J = C_1111 at 16 seeded voxels and its Euler sum.
``batch4`` stores the tangents of the first RVE of each side (64, 128, 256,
512) of the 64-RVE uneven batch.  Workloads with fewer load cases than
strain components store the mean stresses and each solve's residual history.
``spheres128`` is solved one load case per process (``spheres128:<l>``, each
writes ``spheres128_lc<l>.json``); ``spheres128:merge`` assembles
``spheres128.json`` from the six parts.  Nothing here calls the CUDA path.
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
TOL = 1e-12
SOURCE = "oracle.fe_projection.Problem (O1), FP64, scipy FFT of the real fields"


def _run(name):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    import numpy as np

    import microstructures as ms
    from oracle.fe_projection import Problem

    if name.startswith("spheres128:"):
        part = name.split(":", 1)[1]
        if part == "merge":
            parts = [json.load(open(os.path.join(HERE, f"spheres128_lc{l}.json"))) for l in range(6)]
            S = np.array([p["mean_stress"] for p in parts])     # S[l][:] for unit strain e_l
            out = dict(name="spheres128", n=parts[0]["n"], nu=parts[0]["nu"], tol=TOL,
                       source=parts[0]["source"], C_eff=S.T.tolist(),
                       iterations=[p["iterations"] for p in parts],
                       seconds=sum(p["seconds"] for p in parts))
            with open(os.path.join(HERE, "spheres128.json"), "w") as f:
                json.dump(out, f, indent=1)
            return name
        l = int(part)
        cfg = ms.config_inputs("spheres128")
        t0 = time.time()
        P = Problem(cfg["n"], cfg["E"], cfg["nu"])
        eps, it, res = P.solve(np.eye(6)[l], tol=TOL)
        out = dict(name=f"spheres128 load case {l}", n=list(cfg["n"]), nu=cfg["nu"], tol=TOL,
                   source=SOURCE,
                   mean_stress=P.mean_stress(eps).tolist(), iterations=it, rel_residual=float(res),
                   seconds=time.time() - t0)
        with open(os.path.join(HERE, f"spheres128_lc{l}.json"), "w") as f:
            json.dump(out, f, indent=1)
        return name

    if name == "batch4":
        # the first RVE of each side (64, 128, 256, 512) of the 64-RVE uneven
        # batch, three unit load cases each
        batch = ms.uneven_batch_2d(64, seed=1004)
        picks = {}
        for i, (n, _) in enumerate(batch):
            picks.setdefault(n[0], i)
        t0 = time.time()
        rves = []
        for side in sorted(picks):
            i = picks[side]
            n, E = batch[i]
            C, _, its = Problem(n, E, 0.3).effective_tangent(np.eye(3), tol=TOL)
            rves.append(dict(index=i, n=list(n), C_eff=C.tolist(), iterations=its))
        out = dict(name=name, recipe="microstructures.uneven_batch_2d(64, seed=1004)", nu=0.3, tol=TOL,
                   source=SOURCE, rves=rves, seconds=time.time() - t0)
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        return name

    cfg = ms.config_inputs(name)
    t0 = time.time()
    P = Problem(cfg["n"], cfg["E"], cfg["nu"])
    out = dict(name=name, n=list(cfg["n"]), nu=cfg["nu"], tol=TOL,
               source=SOURCE)
    I = np.eye(P.ns)
    if name == "lognormal64":
        W = np.zeros((P.ns, P.ns)); W[0, 0] = 1.0
        grad, C = P.adjoint_gradient(W, tol=TOL)
        rng = np.random.default_rng(2005)
        vox = rng.choice(grad.size, size=16, replace=False)
        out["adjoint_W"] = W.tolist()
        out["adjoint_voxels"] = [int(v) for v in vox]
        out["adjoint_grad"] = [float(grad.reshape(-1)[v]) for v in vox]
        out["adjoint_euler_sum"] = float(np.sum(P.E * grad))
        out["C_eff"] = C.tolist()
    else:
        Em = cfg["E_macro"]
        if len(Em) == P.ns:
            C, fields, its = P.effective_tangent(Em, tol=TOL)
            out["C_eff"] = C.tolist()
            out["iterations"] = its
        else:
            S = []
            its = []
            hists = []
            for row in Em:
                hist = []
                eps, it, _ = P.solve(row, tol=TOL, history=hist)
                S.append(P.mean_stress(eps).tolist())
                its.append(it)
                hists.append(hist)
            out["mean_stress"] = S
            out["iterations"] = its
            # ||r_k|| / ||r_0|| for k = 0..iterations: how many iterations the
            # oracle needs for a looser tolerance
            out["rel_residual_history"] = hists
        if name == "disc32":
            from oracle.fem_assembly import AssembledFEM
            C2, _ = AssembledFEM(cfg["n"], cfg["E"], cfg["nu"]).effective_tangent(I)
            out["C_eff_fem"] = C2.tolist()
            Cf, _, its = P.effective_tangent(I, tol=TOL)
            out["C_eff"] = Cf.tolist()
            out["iterations_unit"] = its
    out["seconds"] = time.time() - t0
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    return name


if __name__ == "__main__":
    names = sys.argv[1:] or ["disc32", "gauss1024", "lognormal64"]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(names)) as pool:
        for n in pool.imap_unordered(_run, names):
            print("wrote", n, flush=True)
