"""The C-ABI library loads and exports every entry point include/*.h declares;
host-side argument checks (no GPU work)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2404_02628_gb300 import build

    build.build()
    import paper_2404_02628_gb300 as p

    p.load()
    return p


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pimd_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(pkg):
    names = declared_functions()
    assert len(names) >= 20
    L = pkg.load()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(pkg.symbols()) <= names


def test_binding_covers_header(pkg):
    assert declared_functions() <= set(pkg.symbols())


def test_create_rejects_bad_arguments(pkg):
    bad = [(0, 4, 2, 1.0, 1.0, 0.0, 0.5, 1.0), (4, 1, 2, 1.0, 1.0, 0.0, 0.5, 1.0),
           (4, 4, 4, 1.0, 1.0, 0.0, 0.5, 1.0), (4, 4, 2, 0.0, 1.0, 0.0, 0.5, 1.0),
           (4, 4, 2, 1.0, 1.0, 0.0, 0.0, 1.0), (4, 4, 2, 1.0, 1.0, 0.0, 0.5, 1.5),
           (4, 4, 2, 1.0, 1.0, 0.0, 0.5, -0.1), (4, 4, 2, 1.0, -1.0, 0.0, 0.5, 1.0)]
    for args in bad:
        with pytest.raises(pkg.PimdError) as ei:
            pkg.pimd_create(*args)
        assert ei.value.status == pkg.PIMD_EINVAL


def test_config_and_workspace_host_logic(pkg):
    h = pkg.pimd_create(1000, 8, 2, 2.0, 1.0, 3.0, 0.5, 1.0)
    try:
        cfg = pkg.pimd_default_config()
        assert cfg.dt == 0.01 and cfg.nhc_len == 4 and cfg.thermostat == 1
        cfg.nhc_len = 0
        with pytest.raises(pkg.PimdError):
            pkg.pimd_configure(h, cfg)
        cfg.nhc_len = 4
        pkg.pimd_configure(h, cfg)
        with pytest.raises(pkg.PimdError):
            pkg.pimd_workspace_bytes(h, 1000)  # not a multiple of 32
        n_store = pkg.pimd_workspace_bytes(h, 1024)
        cfg.table_mode = pkg.TABLE_RECOMPUTE
        pkg.pimd_configure(h, cfg)
        n_rec = pkg.pimd_workspace_bytes(h, 1024)
        assert n_rec < n_store
        # state calls before bind are refused
        with pytest.raises(pkg.PimdError) as ei:
            pkg.pimd_step(h, 1)
        assert ei.value.status == pkg.PIMD_ESTATE
    finally:
        pkg.pimd_destroy(h)


def test_workspace_scales_quadratically_in_store_mode(pkg):
    def ws(N, mode):
        h = pkg.pimd_create(N, 32, 2, 3.0, 1.0, 0.0, 0.5, 1.0)
        cfg = pkg.pimd_default_config()
        cfg.table_mode = mode
        pkg.pimd_configure(h, cfg)
        n = pkg.pimd_workspace_bytes(h, (N + 31) // 32 * 32)
        pkg.pimd_destroy(h)
        return n

    a, b = ws(10000, pkg.TABLE_STORE), ws(40000, pkg.TABLE_STORE)
    assert 14 < b / a < 18
    c, d = ws(10000, pkg.TABLE_RECOMPUTE), ws(40000, pkg.TABLE_RECOMPUTE)
    assert d / c < 5 and d < 0.02 * b


def test_batch_create_rejects_bad_arguments(pkg):
    bad = [([0, 5], [1.0, 1.0], [1.0, 1.0]), ([2048, 5], [1.0, 1.0], [1.0, 1.0]),
           ([4, 5], [0.0, 1.0], [1.0, 1.0]), ([4, 5], [1.0, 1.0], [1.0, 1.5]),
           ([4, 5], [1.0, 1.0], [-0.2, 1.0])]
    for Ns, betas, xis in bad:
        with pytest.raises(pkg.PimdError) as ei:
            pkg.pimd_batch_create(Ns, 4, 2, betas, xis, 1.0, 0.0, 0.5)
        assert ei.value.status == pkg.PIMD_EINVAL


def test_batch_layout_and_workspace_host_logic(pkg):
    Ns = [1, 31, 32, 33, 500]
    P, d = 8, 2
    h = pkg.pimd_batch_create(Ns, P, d, [1.0, 2.0, 3.0, 4.0, 1.0], [1.0, 0.0, 0.5, 1.0, 1.0], 1.0, 3.0, 0.5)
    try:
        off = pkg.pimd_batch_layout(h, len(Ns))
        pads = [(n + 31) // 32 * 32 for n in Ns]
        assert off[0] == 0
        assert [off[i + 1] - off[i] for i in range(len(Ns))] == [P * d * n for n in pads]
        small = pkg.pimd_batch_workspace_bytes(h)
        cfg = pkg.pimd_default_config()
        cfg.nhc_len = 0
        with pytest.raises(pkg.PimdError):
            pkg.pimd_batch_configure(h, cfg)
    finally:
        pkg.pimd_batch_destroy(h)
    h = pkg.pimd_batch_create(Ns + [2047], P, d, [1.0] * 6, [1.0] * 6, 1.0, 3.0, 0.5)
    try:
        big = pkg.pimd_batch_workspace_bytes(h)
        # the stored factor table of the 2047-particle replica alone is ~64*65/2 tiles of 12 KB
        assert big > small + 64 * 65 // 2 * 12288
    finally:
        pkg.pimd_batch_destroy(h)


def test_vb_table_mode_and_workspace(pkg):
    """pimd_vb: automatic store up to N = 16383, recompute above (O(N) workspace)."""
    sizes = {}
    for N in (10000, 16383, 16384, 20000, 30000, 40000):
        h = pkg.pimd_vb_create(N, 32, 2, 3.0, 1.0)
        try:
            sizes[N] = pkg.pimd_vb_workspace_bytes(h)
            if N == 10000:
                pkg.pimd_vb_set_table_mode(h, pkg.TABLE_RECOMPUTE)
                small = pkg.pimd_vb_workspace_bytes(h)
                assert small < sizes[N] / 10
                pkg.pimd_vb_set_table_mode(h, -1)
                assert pkg.pimd_vb_workspace_bytes(h) == sizes[N]
                with pytest.raises(pkg.PimdError):
                    pkg.pimd_vb_set_table_mode(h, 7)
        finally:
            pkg.pimd_vb_destroy(h)
    assert sizes[16383] > 12 * 16383 * 16384 // 2          # stored table
    assert sizes[16384] < sizes[16383] / 20                 # recomputed
    assert sizes[40000] < 12 * 40000 * 40001 // 2 // 50     # O(N): 127 MB against the 9.6 GB table
    assert sizes[20000] < sizes[30000] < sizes[40000]


def test_autotune_requires_bound_handle(pkg):
    h = pkg.pimd_create(100, 4, 2, 1.0, 1.0, 0.0, 0.5, 1.0)
    try:
        with pytest.raises(pkg.PimdError) as ei:
            pkg.pimd_autotune(h, None)
        assert ei.value.status == pkg.PIMD_ESTATE
    finally:
        pkg.pimd_destroy(h)
    b = pkg.pimd_batch_create([10, 20], 4, 2, [1.0, 1.0], [1.0, 1.0], 1.0, 0.0, 0.5)
    try:
        with pytest.raises(pkg.PimdError) as ei:
            pkg.pimd_batch_autotune(b, None)
        assert ei.value.status == pkg.PIMD_ESTATE
    finally:
        pkg.pimd_batch_destroy(b)


def test_init_state_and_density_require_bound_handle(pkg):
    """Host-side checks of the seeded initial state and the density estimator
    (no device work: the handle is never bound)."""
    h = pkg.pimd_create(100, 4, 2, 1.0, 1.0, 0.0, 0.5, 1.0)
    try:
        for call in (lambda: pkg.pimd_init_state(h, 1), lambda: pkg.pimd_density_accumulate(h, 16, 3.0, 1 << 20)):
            with pytest.raises(pkg.PimdError) as ei:
                call()
            assert ei.value.status == pkg.PIMD_ESTATE
        with pytest.raises(pkg.PimdError) as ei:
            pkg.pimd_density_accumulate(h, 16, 3.0, 0)  # NULL histogram
        assert ei.value.status == pkg.PIMD_EINVAL
    finally:
        pkg.pimd_destroy(h)
    b = pkg.pimd_batch_create([10, 20], 4, 2, [1.0, 1.0], [1.0, 1.0], 1.0, 0.0, 0.5)
    try:
        with pytest.raises(pkg.PimdError) as ei:
            pkg.pimd_batch_init_state(b, 7)
        assert ei.value.status == pkg.PIMD_ESTATE
    finally:
        pkg.pimd_batch_destroy(b)


def test_batch_tuning_host_query(pkg):
    b = pkg.pimd_batch_create([10, 20], 4, 2, [1.0, 1.0], [1.0, 1.0], 1.0, 3.0, 0.5)
    try:
        t = pkg.pimd_batch_tuning(b)
        assert t["pair_block"] in (64, 128, 256)
    finally:
        pkg.pimd_batch_destroy(b)


def test_species_host_logic(pkg):
    """pimd_set_species: counts must be positive and add up to N, at most four
    species, only before bind; the workspace holds one exchange region per
    species (smaller in store mode, since N_A^2 + N_B^2 < N^2)."""
    h = pkg.pimd_create(1000, 8, 2, 2.0, 1.0, 3.0, 0.5, 1.0)
    try:
        one = pkg.pimd_workspace_bytes(h, 1024)
        for bad in ([500, 499], [0, 1000], [200] * 5, [1001]):
            with pytest.raises(pkg.PimdError) as ei:
                pkg.pimd_set_species(h, bad)
            assert ei.value.status == pkg.PIMD_EINVAL
        pkg.pimd_set_species(h, [400, 600])
        two = pkg.pimd_workspace_bytes(h, 1024)
        assert 0 < two < one
        pkg.pimd_set_species(h, [1000])
        assert pkg.pimd_workspace_bytes(h, 1024) == one
    finally:
        pkg.pimd_destroy(h)
