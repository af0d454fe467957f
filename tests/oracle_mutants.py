"""Plants one plausible mistake at a time in a copy of the oracle and runs the CPU
pins (tests/test_oracle_*.py, the conditioning measurements excluded) against it:
every mutant must fail at least one pin.  Not collected by pytest (minutes per
mutant); run by hand:

    python tests/oracle_mutants.py [scratch directory]
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in oracle/dg2_oracle.c, replacement at its first occurrence)
MUTANTS = [
    ("friction exponent 5/3 for 7/3", "(h * h * cbrt(h))", "(h * cbrt(h))"),
    ("bed-slope sign (Eq. 4a, x)", "- 2.0 * g * U0x.h * z1x / dx;", "+ 2.0 * g * U0x.h * z1x / dx;"),
    ("HLL mass dissipation dropped", "+ sL * sR * (Rs.h - Ls.h)) / den", ") / den"),
    ("Eq. 4b factor 3 -> 2 (x)", "real L1xh = -(3.0 / dx)", "real L1xh = -(2.0 / dx)"),
    ("minmod takes the max", "return m < c ? m : c;", "return m > c ? m : c;"),
    ("inflow discharge per face, not per width", "/ (nf * d);", "/ (nf);"),
    ("half the rain", "if (raining) L0h += o->rain;", "if (raining) L0h += 0.5 * o->rain;"),
    ("point source per dx only", "L0h += o->qp / (dx * dy);", "L0h += o->qp / dx;"),
    ("dry reset keeps discharges", "for (int k = 1; k < 9; ++k) U[k * N + c] = 0.0;",
     "for (int k = 1; k < 3; ++k) U[k * N + c] = 0.0;"),
    ("y flux: u for v in the mass flux", "return mk(s.h * v, s.h * u * v,",
     "return mk(s.h * u, s.h * u * v,"),
    ("gauge xi over dx, not dx / 2", "double xi = (x - (i + 0.5) * o->dx) / (0.5 * o->dx)",
     "double xi = (x - (i + 0.5) * o->dx) / o->dx"),
    ("gauge eta scaled by dx", "et = (y - (j + 0.5) * o->dy) / (0.5 * o->dy)",
     "et = (y - (j + 0.5) * o->dy) / (0.5 * o->dx)"),
    ("gauge depth not clipped", "    return h > 0.0 ? h : 0.0;\n}\n\n/* Advances to t_end",
     "    return h;\n}\n\n/* Advances to t_end"),
]


def run(scratch):
    survivors = []
    for k, (name, old, new) in enumerate(MUTANTS):
        tree = os.path.join(scratch, f"mutant{k}")
        shutil.rmtree(tree, ignore_errors=True)
        skip = shutil.ignore_patterns("__pycache__", "*.so")
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(tree, "tests"), ignore=skip)
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tree, "oracle"), ignore=skip)
        pkg = os.path.join(tree, "paper_2010_02003_gb300")
        os.makedirs(pkg)
        for f in ("__init__.py", "inputs.py"):
            shutil.copy(os.path.join(ROOT, "paper_2010_02003_gb300", f), pkg)
        src = os.path.join(tree, "oracle", "dg2_oracle.c")
        text = open(src).read()
        assert old in text, name
        open(src, "w").write(text.replace(old, new, 1))
        r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "not gpu", "-q", "-p",
                            "no:cacheprovider", "-k", "oracle and not conditioning"],
                           cwd=tree, capture_output=True, text=True)
        failed = [l.split("::")[-1] for l in r.stdout.splitlines() if l.startswith("FAILED")]
        print(f"{name}: {len(failed)} pins fail {failed[:3]}", flush=True)
        if not failed:
            survivors.append(name)
        shutil.rmtree(tree, ignore_errors=True)
    return survivors


if __name__ == "__main__":
    scratch = sys.argv[1] if len(sys.argv) > 1 else tempfile.mkdtemp(prefix="oracle_mutants_")
    left = run(scratch)
    print("surviving mutants:", left)
    sys.exit(1 if left else 0)
