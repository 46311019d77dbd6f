"""Full-size certification of the library's solves by the FP64 oracle (a script beside the
tests; it runs a GPU solve, then the oracle on the host).

    python tests/certify.py NAME [--out FILE]      NAME in mbb_c1 mbb_c2 mbb_c3 mbb_c5
                                                   cantilever_batch

For every realisation (every instance of the batch) the library solves K(E_k) u_k = f in
MIXED precision to a true relative residual of 1e-8, exactly as the benchmark does.  The
oracle then, independently of the library:
  - runs its own design chain (filter, projection, SIMP) to get E_k;
  - forms the residual ||f - K(E_k) u_k||_2 / ||f||_2 over the free DOFs with its own
    element-by-element operator (the definition of Sec. 2.1), and, up to 4.2M DOFs, with its
    assembled CSR matrix as well;
  - recomputes the compliance f^T u_k (Sec. 2.2) and compares it with the library's;
  - on the 192x64 and 1024x512 workloads (and four seeded instances of the batch) solves
    the system by sparse LU and reports the energy-norm error of u_k (Sec. 3.1) and the
    compliance against the direct solution.
Prints one JSON line (and writes it to --out).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import fem, msfem, pipeline  # noqa: E402

DIRECT = {"mbb_c1", "mbb_c2"}
CSR_LIMIT = 4_300_000


def gpu_solve(wl):
    import torch
    import paper_1411_3923_gb300 as m
    prob = m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                     penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision="mixed", tol=wl.tol,
                     max_iter=5000)
    prob.set_design(torch.from_numpy(np.ascontiguousarray(wl.rho)).cuda(), wl.rmin, wl.beta,
                    wl.etas, wl.cell)
    info = prob.build_preconditioner()
    u, infos = prob.solve(torch.from_numpy(np.ascontiguousarray(wl.force)).cuda(), -1)
    u = u.cpu().numpy()
    prob.close()
    return u, infos, info


def certify(wl, direct: bool):
    t0 = time.time()
    u, infos, binfo = gpu_solve(wl)
    t_gpu = time.time() - t0
    grid, K0, prob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"]
    f_or = grid.nodal_from_neutral(wl.force)
    ff = f_or[prob.free]
    nf = np.linalg.norm(ff)
    rows = []
    for k in range(len(wl.etas)):
        row = {"realisation": k, "eta": wl.etas[k], "status": infos[k]["status"],
               "iterations": infos[k]["iterations"],
               "library_rel_residual": infos[k]["rel_residual"]}
        y = prob.apply(E[k], u[k])                       # element by element, fixed rows zero
        r = ff - grid.nodal_from_neutral(y)[prob.free]
        row["oracle_rel_residual"] = float(np.linalg.norm(r) / nf)
        uf = grid.nodal_from_neutral(u[k])[prob.free]
        if grid.n_dof <= CSR_LIMIT:
            Kf = prob.free_matrix(E[k])
            row["oracle_csr_rel_residual"] = float(np.linalg.norm(ff - Kf @ uf) / nf)
        c_or = float(ff @ uf)
        row["compliance"] = infos[k]["compliance"]
        row["compliance_oracle_f_dot_u_rel_diff"] = abs(infos[k]["compliance"] / c_or - 1.0)
        if direct:
            ud = prob.solve_direct(E[k], wl.force)
            udf = grid.nodal_from_neutral(ud)[prob.free]
            Kf = prob.free_matrix(E[k])
            c_d = float(ff @ udf)
            row["direct_compliance"] = c_d
            row["compliance_rel_err_vs_direct"] = abs(infos[k]["compliance"] / c_d - 1.0)
            row["energy_error_vs_direct"] = msfem.energy_error(Kf, udf, uf)
        rows.append(row)
    return {"mesh": [wl.nelx, wl.nely], "dofs": grid.n_dof, "realisations": len(wl.etas),
            "gpu_s": round(t_gpu, 2), "oracle_s": round(time.time() - t0 - t_gpu, 2),
            "n_types": binfo["n_types"], "n_coarse": binfo["n_coarse"], "systems": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=["mbb_c1", "mbb_c2", "mbb_c3", "mbb_c5", "cantilever_batch"])
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = {"certify": args.name, "tol": 1e-8, "precision": "mixed"}
    if args.name == "cantilever_batch":
        wls = workloads.cantilever_batch()
        rng = np.random.default_rng(44)
        with_direct = set(int(i) for i in rng.choice(len(wls), 4, replace=False))
        inst = []
        for b, wl in enumerate(wls):
            c = certify(wl, b in with_direct)
            c["instance"] = b
            inst.append(c)
        out["instances"] = inst
        out["dofs"] = sum(c["dofs"] for c in inst)
        sy = [s for c in inst for s in c["systems"]]
    else:
        wl = workloads.make(args.name)
        out.update(certify(wl, args.name in DIRECT))
        sy = out["systems"]
    out["worst_oracle_rel_residual"] = max(s["oracle_rel_residual"] for s in sy)
    out["all_converged"] = all(s["status"] == 0 for s in sy)
    if any("energy_error_vs_direct" in s for s in sy):
        out["worst_energy_error_vs_direct"] = max(s.get("energy_error_vs_direct", 0.0) for s in sy)
        out["worst_compliance_rel_err_vs_direct"] = max(
            s.get("compliance_rel_err_vs_direct", 0.0) for s in sy)
    line = json.dumps(out)
    print(line)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(line + "\n")


if __name__ == "__main__":
    main()
