"""Write kirkwood_sphere_r10_100sites.json: the closed-form Delta G_solv of the 100
multipole sites of the R = 10 A sphere workload (Kirkwood's series for a dielectric
sphere in a screened solvent, extended to point quadrupoles and Thole-damped induced
dipoles; ``oracle.kirkwood.solvation``), together with a digest of the sites it was
computed for.  The GPU tests at 20,480 panels read it instead of spending ~20 s on
the series.  Run from the repository root: python tests/golden/make_kirkwood_sphere_r10.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import gen  # noqa: E402
from oracle import kirkwood  # noqa: E402

OUT = os.path.join(HERE, "kirkwood_sphere_r10_100sites.json")


def sites_digest(sites) -> str:
    h = hashlib.sha256()
    for a in (sites.pos, sites.q, sites.d, sites.Q, sites.alpha):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


def main():
    pr = gen.sphere_r10_20480()
    p = pr.params
    dG, mu, mu_v = kirkwood.solvation(pr.sites, 10.0, p.eps_in, p.eps_out, p.kappa, p.thole_a)
    rec = {"what": "closed-form Delta G_solv (kcal/mol) of gen.sphere_r10_20480's sites in a sphere of radius "
                   "10 A, eps_in 1, eps_out 80, kappa 0.125 1/A, Thole a 0.39 (oracle.kirkwood.solvation)",
           "radius": 10.0, "eps_in": p.eps_in, "eps_out": p.eps_out, "kappa": p.kappa, "thole_a": p.thole_a,
           "n_sites": int(pr.sites.n), "sites_sha256": sites_digest(pr.sites), "dG_kcal": float(dG)}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
