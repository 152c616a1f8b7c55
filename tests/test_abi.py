"""The C-ABI library loads and exports every entry point include/mfa.h declares (no GPU needed)."""

import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mfa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mfa_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("mfa_encode_blocks", "mfa_decode_blocks", "mfa_raycast", "mfa_adjoint_blocks"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2409_00184_b300 import build
    import ctypes
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2409_00184_b300 import mfa
    assert sorted(mfa.SYMBOLS) == _declared()


def test_descriptor_layout_matches_header():
    from paper_2409_00184_b300 import mfa
    assert mfa.DESC_DTYPE.itemsize == 72
    assert mfa.DESC_DTYPE.fields["knot_off"][1] == 40 and mfa.DESC_DTYPE.fields["cp_off"][1] == 64


def test_model_bytes_eq2_golden():
    from paper_2409_00184_b300 import mfa
    rows = np.loadtxt(os.path.join(ROOT, "tests", "golden", "eq2_model_size.txt"), dtype=np.int64)
    for ncp, deg, size in rows:
        assert mfa.model_bytes(int(ncp), int(deg)) == size
    assert mfa.model_bytes(0, 2) == -1


def test_struct_mirrors_match_the_library():
    """The ctypes structs of the binding have the sizes the library was compiled with (a field added to a
    C struct without its mirror, or the other way round, fails here)."""
    import ctypes
    from paper_2409_00184_b300 import mfa
    want = [ctypes.sizeof(t) for t in (mfa.BlockDesc, mfa.Bounds, mfa.DecodeTiling, mfa.View, mfa.FrameDesc)]
    assert mfa.abi_struct_sizes() == want


def test_product_code_never_reaches_the_oracle():
    """The package (binding, autograd, adaptive encoding, out-of-core sequencing, build) and the library
    sources name no oracle module: every result of the product path comes from the CUDA library. The oracle
    and the library share no source either (the oracle is plain numpy)."""
    pkg = os.path.join(ROOT, "paper_2409_00184_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\b(import|from)\s+oracle\b|oracle\.", src), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2409_00184_b300" not in src and "libmfa" not in src, f
    # the seeded input generators serve both sides and import neither
    src = open(os.path.join(ROOT, "synth", "__init__.py")).read()
    assert not re.search(r"\b(import|from)\s+(oracle|paper_2409_00184_b300)\b", src)


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """With libmfa.so missing the binding raises ImportError: there is no CPU or framework fallback."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2409_00184_b300"
    pkg.mkdir()
    for f in ("__init__.py", "mfa.py"):
        shutil.copy(os.path.join(ROOT, "paper_2409_00184_b300", f), pkg / f)
    r = subprocess.run([sys.executable, "-c", "import paper_2409_00184_b300.mfa"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "ImportError" in r.stderr and "no fallback" in r.stderr


def _undocumented(lines):
    """Functions whose declaration is not reached, walking up without crossing a blank line, from the end of
    a comment block (their own, or the one opening their group of declarations and flag defines)."""
    out = []
    for i, line in enumerate(lines):
        m = re.match(r"\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(mfa_[a-z_0-9]+)\s*\(", line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and lines[j].strip() and not lines[j].rstrip().endswith("*/"):
            j -= 1
        if j < 0 or not lines[j].rstrip().endswith("*/"):
            out.append(m.group(1))
    return out


def test_every_entry_point_is_documented():
    """Every function include/mfa.h declares sits under a comment (its own, or one shared with the
    declarations right after it), which states what it computes, its arguments and its errors."""
    probe = ["/* a */", "int mfa_a(int x);", "", "int mfa_b(int y);", "/* c, d */", "int mfa_c(void);",
             "#define X 1", "int mfa_d(void);"]
    assert _undocumented(probe) == ["mfa_b"]  # the check itself
    lines = open(os.path.join(ROOT, "include", "mfa.h")).read().splitlines()
    assert not _undocumented(lines), _undocumented(lines)
