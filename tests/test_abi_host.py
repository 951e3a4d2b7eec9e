"""CPU-only checks of the C ABI: the library loads, exports every symbol that
include/*.h declares, and its host-side planner (the structural dry run)
groups terms and orders offsets bit-exactly like the oracle."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_2606_16959_gb300 import hs, workloads as W


def declared_symbols():
    """Every entry point declared in include/*.h."""
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|void|uint64_t|const char\*)\s+(hs_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2606_16959_gb300 import _build
    _build.build()
    return hs.lib()


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(hs.EXPORTS) == decl


def test_debug_bounds_word_of_ordinary_build(lib):
    """The ordinary build has no index checks: hs_debug_bounds says so without
    touching a device, and rejects a null output."""
    if hs.DEBUG_BOUNDS:
        pytest.skip("the index-checking build is loaded")
    assert hs.hs_debug_bounds() is None
    assert lib.hs_debug_bounds(None, 0) == hs.HS_EINVAL


def test_debug_bounds_sources():
    """Every kernel translation unit that addresses factor values, tables or
    states goes through the index check of the HS_DEBUG_BOUNDS build."""
    csrc = os.path.join(ROOT, "paper_2606_16959_gb300", "csrc")
    sites = {}
    for name in ("sweep_core.cuh", "apply.cu", "qsweep.cu", "build.cu", "dia.cu"):
        sites[name] = set(re.findall(r"BS_[A-Z_]+", open(os.path.join(csrc, name)).read()))
    used = set().union(*sites.values())
    declared = set(re.findall(r"^\s*(BS_[A-Z_]+)\s*=", open(os.path.join(csrc, "bounds.cuh")).read(), flags=re.M))
    assert declared and used == declared, (declared - used, used - declared)


def test_plan_rejects_bad_input(lib):
    with pytest.raises(hs.HSError) as e:
        hs.hs_plan_factors([1], [0], 0, 4)
    assert e.value.code == hs.HS_EINVAL
    with pytest.raises(hs.HSError):
        hs.hs_plan_factors([1], [0], 4, 0)
    with pytest.raises(hs.HSError):
        hs.hs_plan_factors([1 << 5], [0], 4, 4)  # mask beyond n_qubits
    with pytest.raises(hs.HSError):
        hs.hs_plan_factors([(1 << 13) - 1], [0], 13, 4)  # 13 flipped qubits: over 4096 diagonals


def _value_table_entries(x, z, group, n_diags):
    """Entries of a factor's value table: |X| slots times 2^(index bits), for
    factors with slot tables (<= 32 diagonals) touching <= 8 qubits.  The index
    bits are the qubits the terms touch, or the window of consecutive qubits
    covering them when it is at most 8 wide with at most two gaps."""
    first, last = group
    if n_diags > 32:
        return 0
    support = 0
    span = set([0])
    for j in range(first, last):
        support |= int(x[j]) | int(z[j])
        span |= {u ^ int(x[j]) for u in span}
    bits = bin(support).count("1")
    if support:
        lo = (support & -support).bit_length() - 1
        width = support.bit_length() - lo
        if width <= 8 and width <= bits + 2:
            bits = width
    entries = len(span) << bits
    return entries if bits <= 8 and entries <= 2048 else 0


def _compare(oracle, x, z, n, budget):
    got, vbytes = hs.hs_plan_factors(x, z, n, budget)
    want = oracle.group_terms(x, budget)
    assert [(g[0], g[1]) for g in got] == [(g.first, g.last) for g in want]
    for g, w in zip(got, want):
        assert g[2] == w.offsets
    N = 1 << n
    S = sum(N - abs(d) for g in got for d in g[2])
    V = sum(_value_table_entries(x, z, (g[0], g[1]), len(g[2])) for g in got)
    assert (S + V) * 8 <= vbytes <= (S + V + 4 * sum(len(g[2]) for g in got) + 4) * 8


def test_plan_matches_oracle_families(oracle, lib):
    for ham, budgets in [(W.tfim_chain(10, 1, 1), (1, 3, 4, 8)), (W.heisenberg_chain(16, np.ones(16)), (4, 5, 8, 16)),
                         (W.maxcut_3regular(24, 1003), (1, 4, 9)), (W.tsp_onehot(4, 5), (1,)),
                         (W.tfim_chain(20, 1, 1, periodic=True), (4, 7, 16))]:
        x, z, n = oracle.parse_terms(ham.labels)
        for b in budgets:
            _compare(oracle, x, z, n, b)


def test_plan_matches_oracle_random(oracle, lib):
    rng = np.random.default_rng(77)
    for trial in range(200):
        n = int(rng.integers(1, 12))
        m = int(rng.integers(1, 14))
        labels = ["".join(rng.choice(list("IXYZ"), p=[0.55, 0.15, 0.15, 0.15], size=n)) for _ in range(m)]
        x, z, _ = oracle.parse_terms(labels)
        _compare(oracle, x, z, n, int(rng.integers(1, 24)))


def test_batch_and_serve_generators_plan(oracle, lib):
    for job in W.batch256(n_jobs=24, n_hi=14):
        x, z, n = oracle.parse_terms(job.ham.labels)
        _compare(oracle, x, z, n, job.budget)


def test_parse_terms_matches_oracle(oracle, lib):
    """Term canonicalisation in the library (hs_parse_terms) equals the oracle's parser bit for bit."""
    rng = np.random.default_rng(78)
    for trial in range(100):
        n = int(rng.integers(1, 31))
        labels = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(int(rng.integers(1, 20)))]
        x, z, nq = hs.hs_parse_terms(labels)
        ox, oz, on = oracle.parse_terms(labels)
        assert nq == on and np.array_equal(x, np.asarray(ox, np.uint64)) and np.array_equal(z, np.asarray(oz, np.uint64))
    for bad in (["XQ"], ["XX", "X"], [], ["I" * 31]):
        with pytest.raises(hs.HSError) as e:
            hs.hs_parse_terms(bad)
        assert e.value.code == hs.HS_EINVAL


def test_no_pauli_parsing_in_python_package():
    """Labels are parsed only by the library: the Python package marshals them."""
    pkg = os.path.join(ROOT, "paper_2606_16959_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert 'in "XY"' not in src and 'in "ZY"' not in src, name
