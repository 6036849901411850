"""Mutation sweep of the oracle's pins (test infrastructure, CPU only).

Plants one small mistake at a time in ``gs_oracle.c`` (a flipped sign or
operator, an off-by-one comparison or bound, a swapped index, a changed
constant, ``&&`` for ``||``) or, with ``--target optim.py``, in the Adam and
loss reference, rebuilds the oracle in a scratch copy and runs the oracle's pin
tests (``tests/test_oracle_*.py``) against it.  A mutant the
pins do not catch ("survives") is either equivalent to the original, or marks a
part of the oracle no pin fixes yet.  Comments, docstrings and preprocessor lines
are never mutated.  Nothing of the CUDA library is involved.

    python oracle/mutation_sweep.py [--target gs_oracle.c|optim.py] [--jobs 6] [--out survivors.txt]

Scratch copies go under ``oracle/_build/mutants``.  A full sweep is about 700
mutants, a few minutes on 8 cores.
"""
from __future__ import annotations

import argparse
import os
import queue
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SCRATCH = os.path.join(HERE, "_build", "mutants")

# (pattern, replacement): each match of a pattern in a code span is one mutant
OPERATORS = [
    (r" \+ ", " - "), (r" - ", " + "), (r" \* ", " / "),
    (r"(?<=[^<>=!])<(?=[^<=])", "<="), (r"<=", "<"), (r"(?<=[^<>=-])>(?=[^>=])", ">="), (r">=", ">"),
    (r"\[0\]", "[1]"), (r"\[1\]", "[0]"), (r"\[2\]", "[1]"),
    (r"(?<![\w.])2\.0(?![\w.])", "1.0"), (r"(?<![\w.])0\.5(?![\w.])", "0.25"),
    (r"(?<![\w.])3\.0(?![\w.])", "2.0"), (r"(?<![\w.])1\.0(?![\w.])", "2.0"),
    (r"\+= ", "-= "), (r"-= ", "+= "), (r"\+ 1\b", "+ 0"), (r"- 1\b", "- 0"),
    (r"&&", "||"), (r"\|\|", "&&"),
    (r"\bfloor\(", "ceil("), (r"\bfmin\(", "fmax("), (r"\bfmax\(", "fmin("), (r"\bexp\(-", "exp("),
    (r"\bsqrt\(", "fabs("), (r"\[3\]", "[2]"),
]
# Python only: powers, square roots, the sigmoid derivative's factor
PY_OPERATORS = [(r"\*\*", "*"), (r"np\.sqrt", "np.abs"), (r"\(1 - o\)", "(1 + o)"), (r"\(1 - b", "(1 + b")]


def code_spans(lines):
    """Per line, the column spans that are C code (outside comments and
    preprocessor lines)."""
    out = []
    in_block = False
    for ln in lines:
        spans = []
        if not in_block and ln.lstrip().startswith("#"):
            out.append(spans)
            continue
        i = 0
        while i < len(ln):
            if in_block:
                j = ln.find("*/", i)
                if j < 0:
                    break
                in_block = False
                i = j + 2
                continue
            jb, jl = ln.find("/*", i), ln.find("//", i)
            starts = [x for x in (jb, jl) if x >= 0]
            j = min(starts) if starts else len(ln)
            if j > i:
                spans.append((i, j))
            if j == len(ln) or j == jl:
                break
            in_block = True
            i = j + 2
        out.append(spans)
    return out


def python_code_spans(lines):
    """Per line, the column spans that are Python code (outside docstrings,
    comments and import lines)."""
    out = []
    in_doc = False
    for ln in lines:
        st = ln.strip()
        quotes = ln.count('"""')
        if in_doc or quotes:
            out.append([])
            in_doc = in_doc != (quotes % 2 == 1)
            continue
        if st.startswith(("#", "import ", "from ")):
            out.append([])
            continue
        j = ln.find("#")
        out.append([(0, j if j >= 0 else len(ln))])
    return out


def mutants(text: str, first_line: int = 1, python: bool = False):
    """All single-site mutants: (line number, operator pattern, original line, mutated source)."""
    lines = text.split("\n")
    res = []
    ops = OPERATORS + (PY_OPERATORS if python else [])
    for li, spans in enumerate((python_code_spans if python else code_spans)(lines)):
        if li + 1 < first_line:
            continue
        ln = lines[li]
        for a, b in spans:
            for pat, rep in ops:
                for m in re.finditer(pat, ln[a:b]):
                    new = ln[:a + m.start()] + rep + ln[a + m.end():]
                    res.append((li + 1, pat, ln.strip(), "\n".join(lines[:li] + [new] + lines[li + 1:])))
    return res


def _slot(k: int) -> str:
    d = os.path.join(SCRATCH, f"slot{k}")
    if os.path.isdir(d):
        shutil.rmtree(d)
    os.makedirs(d)
    skip = shutil.ignore_patterns("_build", "__pycache__", "*.so", "csrc")
    for sub in ("oracle", "tests", "paper_2312_02121_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=skip)
    return d


def _run(slot: str, target: str, source: str):
    with open(os.path.join(slot, "oracle", target), "w") as f:
        f.write(source)
    shutil.rmtree(os.path.join(slot, "oracle", "_build"), ignore_errors=True)
    tests = sorted(os.path.join("tests", t) for t in os.listdir(os.path.join(slot, "tests"))
                   if t.startswith("test_oracle_") and t.endswith(".py"))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *tests],
                           cwd=slot, env=env, capture_output=True, text=True, timeout=300)
        return p.returncode
    except subprocess.TimeoutExpired:
        return "timeout"  # counts as caught: the pins did not pass


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--target", default="gs_oracle.c", choices=["gs_oracle.c", "optim.py", "__init__.py"])
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--first-line", type=int, default=1, help="mutate only from this source line on")
    ap.add_argument("--out", default="", help="write the surviving mutants here")
    args = ap.parse_args(argv)
    ms = mutants(open(os.path.join(HERE, args.target)).read(), args.first_line, args.target.endswith(".py"))
    print(f"{len(ms)} mutants, {args.jobs} jobs", flush=True)
    free = queue.Queue()
    for k in range(args.jobs):
        free.put(_slot(k))

    def job(m):
        s = free.get()
        try:
            return m, _run(s, args.target, m[3])
        finally:
            free.put(s)

    survivors = []
    with ThreadPoolExecutor(args.jobs) as ex:
        for done, (m, rc) in enumerate(ex.map(job, ms), 1):
            if rc == 0:
                survivors.append(m)
            if done % 50 == 0:
                print(f"{done}/{len(ms)}: {len(survivors)} survive", flush=True)
    report = "".join(f"line {m[0]}: {m[1]!r} in  {m[2]}\n" for m in survivors)
    if args.out:
        with open(args.out, "w") as f:
            f.write(report)
    else:
        sys.stdout.write(report)
    print(f"{len(survivors)} of {len(ms)} mutants survive")
    shutil.rmtree(SCRATCH, ignore_errors=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
