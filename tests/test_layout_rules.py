"""Static checks of the repository's boundaries (CPU only).

The oracle is test infrastructure: the product package (Python binding and
CUDA / C++ sources) neither imports, includes nor links anything under
oracle/, so no product call can fall back to the CPU reference.  Committed
code does not use the scratch folder _work/.
"""

import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2310_11186_gb300")


def _files(base, exts):
    for d, _, names in os.walk(base):
        if "__pycache__" in d or os.sep + "lib" in d[len(base):]:
            continue
        for f in names:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_package_never_uses_the_oracle():
    bad = []
    for path in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        src = open(path, encoding="utf-8").read()
        if re.search(r"^\s*(import|from)\s+oracle\b", src, re.M) or re.search(r'#include\s+"[^"]*oracle', src) \
                or "tsgo_" in src or "libtsgo" in src:
            bad.append(os.path.relpath(path, ROOT))
    assert not bad, bad


def test_committed_code_does_not_use_the_scratch_folder():
    try:
        tracked = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True, check=True).stdout
    except (OSError, subprocess.CalledProcessError):
        tracked = "\n".join(os.path.relpath(p, ROOT) for p in _files(ROOT, (".py", ".cu", ".cuh", ".h", ".c")))
    bad = []
    for rel in tracked.split():
        if not rel.endswith((".py", ".cu", ".cuh", ".h", ".c", ".sh")) or rel.startswith("_work/"):
            continue
        if os.path.abspath(os.path.join(ROOT, rel)) == os.path.abspath(__file__):
            continue  # this file names the folder to look for it
        src = open(os.path.join(ROOT, rel), encoding="utf-8").read()
        if re.search(r"['\"/]_work[/'\"]|\b_work\.", src):
            bad.append(rel)
    assert not bad, bad
