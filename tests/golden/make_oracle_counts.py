"""Write tests/golden/oracle_counts.json: the CPU oracle's FGMRES iteration
count and true relative residual for the named workloads, with the solver
options the benchmark uses (mixed-precision coefficient set, V(nu1,nu2),
FGMRES(m), rel-res 1e-6).  Calls only oracle/ and workloads/.

    python tests/golden/make_oracle_counts.py c1 c2 [--levels L] [--alpha A] [--nu PRE,POST] [--restart M]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import elastic, fgmres, precond  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json")


def auto_levels(n, max_coarse=256):
    L, a, b = 1, n[0], n[1]
    while a * b > max_coarse and a % 2 == 0 and b % 2 == 0 and a // 2 >= 2 and b // 2 >= 2:
        a //= 2
        b //= 2
        L += 1
    return L


def main():
    names = [a for a in sys.argv[1:] if not a.startswith("--")]
    lv = None
    if "--levels" in sys.argv:
        lv = int(sys.argv[sys.argv.index("--levels") + 1])
    al = None
    if "--alpha" in sys.argv:
        al = float(sys.argv[sys.argv.index("--alpha") + 1])
    nu = (1, 2)
    if "--nu" in sys.argv:
        nu = tuple(int(v) for v in sys.argv[sys.argv.index("--nu") + 1].split(","))
    m = 20
    if "--restart" in sys.argv:
        m = int(sys.argv[sys.argv.index("--restart") + 1])
    names = [a for a in names if a not in (str(lv), str(al), ",".join(map(str, nu)), str(m))]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        p = W.config(name)
        L = lv or auto_levels(p.n)
        alpha = al if al is not None else precond.default_alpha(L)
        t0 = time.perf_counter()
        S = elastic.from_problem(p)
        H = S.H
        pc = precond.multigrid(S, L, alpha, precision="mixed", nu_pre=nu[0], nu_post=nu[1])
        b = W.padded_to_compact(W.point_source(p), p.n)
        r = fgmres.fgmres(lambda v: H @ v, b, pc.apply, restart=m, rtol=1e-6, maxit=20000)
        data[name] = {"levels": L, "alpha": alpha, "nu": list(nu), "restart": m, "precision": "mixed", "iters": r.iters,
                      "relres_true": r.relres_true, "converged": bool(r.converged),
                      "cpu_seconds": time.perf_counter() - t0}
        print(name, data[name], flush=True)
        json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
