"""The split of a code over the CTAs of a thread-block cluster (host code of the
cluster and multi-code kernels), compiled with g++ and checked on the CPU: every
check lands on exactly one rank with its variables in row order, every table
entry decodes to the right variable, ranks respect the row cap, and the padding
is what the kernel expects."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_cs_0609090_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_cs_0609090_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("split")
    exe = str(d / "split_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "cluster_split_check.cpp"), "-o", exe],
                   check=True)
    return exe


def _split(exe, code, cs):
    rp = np.asarray(code.row_ptr, np.int32)
    ci = np.asarray(code.col_idx, np.int32)
    W = int(np.diff(rp).max())
    with tempfile.TemporaryDirectory() as d:
        fi, fo = os.path.join(d, "in"), os.path.join(d, "out")
        with open(fi, "wb") as f:
            np.array([code.n_vars, code.n_checks, W, cs], np.int32).tofile(f)
            rp.tofile(f)
            ci.tofile(f)
        subprocess.run([exe, fi, fo], check=True)
        raw = open(fo, "rb").read()
    ok, ns, lb, mr = np.frombuffer(raw[:16], np.int32)
    if not ok:
        return dict(ok=False, ns=int(ns), lb=int(lb))
    o = 16
    rows = np.frombuffer(raw[o:o + 4 * cs], np.int32)
    o += 4 * cs
    rdeg = np.frombuffer(raw[o:o + cs * mr], np.uint8).reshape(cs, mr)
    o += cs * mr
    tab = np.frombuffer(raw[o:o + 2 * cs * W * mr], np.uint16).reshape(cs, W, mr)
    return dict(ok=True, ns=int(ns), lb=int(lb), mr=int(mr), rows=rows, rdeg=rdeg, tab=tab, W=W)


CODES = [("reg36_n1008", lambda: I.make_workload("reg36_n1008", with_llr=False).code),
         ("qc_n7493", lambda: I.make_workload("qc_n7493", with_llr=False).code),
         ("irr_n16200", lambda: I.staircase_code(16200, 5)),
         ("irr_n64800", lambda: I.make_workload("irr_n64800", with_llr=False).code)]


@pytest.mark.parametrize("name,make", CODES, ids=[c[0] for c in CODES])
@pytest.mark.parametrize("cs", [2, 4, 8, 16])
def test_cluster_split(harness, name, make, cs):
    code = make()
    N, M = code.n_vars, code.n_checks
    rp = np.asarray(code.row_ptr)
    ci = np.asarray(code.col_idx)
    t = _split(harness, code, cs)
    ns, lb = t["ns"], t["lb"]
    assert ns % 8 == 0 and ns * cs >= N and (ns - 8) * cs < N
    assert (1 << lb) >= ns
    rb = int(np.ceil(np.log2(cs)))
    if lb + rb > 16:
        assert not t["ok"]
        return
    assert t["ok"]
    mr, rows, rdeg, tab, W = t["mr"], t["rows"], t["rdeg"], t["tab"], t["W"]
    cap = -(-M // cs)
    assert mr % 2 == 0 and mr >= cap and rows.sum() == M and rows.max() <= cap
    want = sorted(tuple(ci[rp[m]:rp[m + 1]]) for m in range(M))
    got = []
    for r in range(cs):
        d = rdeg[r, :rows[r]].astype(int)
        assert np.all(np.diff(d) >= 0)                  # sorted by degree
        assert np.all(rdeg[r, rows[r]:] == 0)           # padding rows
        ent = tab[r, :, :rows[r]].astype(np.int64)
        var = (ent >> lb) * ns + (ent & ((1 << lb) - 1))
        assert np.all((ent >> lb) < cs) and np.all((ent & ((1 << lb) - 1)) < ns)
        for i in range(rows[r]):
            assert np.all(var[d[i]:, i] == var[d[i] - 1, i])  # positions past the degree repeat the last
            got.append(tuple(var[:d[i], i]))
    assert sorted(got) == want
