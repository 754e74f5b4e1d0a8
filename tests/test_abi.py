"""Host-side checks of the C ABI: the library loads, exports every function
``include/pkr.h`` declares, and its host logic (lattice tables, Knudsen map,
argument validation, stability pre-check, memory estimate) agrees with the
oracle and the paper.  No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import lattice, tau_from_knudsen
from oracle.lattice import LATTICES as OR_LATTICES
from oracle.lattice import MAX_ORDER

import __graft_entry__  # noqa: F401  (puts the repo root on the path)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkr():
    from paper_1504_05869_gb300 import build
    build.build()
    import paper_1504_05869_gb300 as pk
    pk._pkr.load()
    return pk


def test_exports_every_declared_symbol(pkr):
    header = open(os.path.join(ROOT, "include", "pkr.h")).read()
    declared = set(re.findall(r"^\s*[\w\s\*]*?\b(pkr_\w+)\s*\(", header, re.M))
    declared = {d for d in declared if not d.endswith("_t")}
    assert declared, "no declarations parsed"
    lib = ctypes.CDLL(pkr._pkr.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(pkr._pkr.EXPORTS)


def test_status_strings(pkr):
    assert pkr._pkr.pkr_status_str(0) == b"ok"
    assert b"unstable" in pkr._pkr.pkr_status_str(-3)
    assert pkr._pkr.pkr_version().startswith(b"pkr")


@pytest.mark.parametrize("name,N", [(n, N) for n in OR_LATTICES for N in (1, 3, 5, 7)
                                    if N <= MAX_ORDER[n]])
def test_library_tables_match_oracle(pkr, name, N):
    """The library's hard-coded and computed tables (its own code) agree with
    the oracle's independently derived ones, velocity by velocity."""
    vel, w, phi, chi, cs2 = pkr.lattice_info(name, N)
    lat = lattice(name, N)
    assert len(w) == lat.Q
    assert abs(cs2 - lat.cs2) <= 2e-16 * lat.cs2
    ref = {tuple(v): (a, b, c) for v, a, b, c in zip(lat.vel, lat.w, lat.phi, lat.chi)}
    assert len({tuple(v) for v in vel}) == lat.Q
    for v, a, b, c in zip(vel, w, phi, chi):
        ra, rb, rc = ref[tuple(int(t) for t in v)]
        assert abs(a - ra) <= 4e-16 * abs(ra)
        # phi/chi are w_i times a polynomial in xi^2 = |v|^2/c_s^2 whose
        # terms reach ~xi^6; both sides round those terms differently
        xi2 = float(np.dot(v, v)) / lat.cs2
        scale = max(ra * (1.0 + xi2 ** 3), abs(rb), abs(rc))
        assert abs(b - rb) <= 4e-16 * scale
        assert abs(c - rc) <= 4e-16 * scale


def test_velocities_grouped_by_class(pkr):
    vel, w, *_ = pkr.lattice_info("D3Q111", 5)
    keys = [tuple(sorted(np.abs(v))[::-1]) for v in vel]
    seen = []
    for k in keys:
        if not seen or seen[-1] != k:
            assert k not in seen, "class split"
            seen.append(k)
    assert len(seen) == 10


def test_tau_from_knudsen_matches_oracle(pkr):
    for name, n in (("D2Q169", (64, 64, 1)), ("D3Q111", (256, 256, 256)),
                    ("D3Q19", (48, 32, 40))):
        for kn in (0.05, 0.1, 0.2, 0.5):
            arr = (ctypes.c_int64 * 3)(*n)
            t = ctypes.c_double()
            assert pkr._pkr.pkr_tau_from_knudsen(pkr.LATTICES[name], kn, arr,
                                                 ctypes.byref(t)) == 0
            assert abs(t.value - tau_from_knudsen(kn, n, lattice(name, 1).cs2)) < 1e-12


def _create(pkr, **kw):
    args = dict(lattice="D3Q111", shape=(8, 8, 8), order=5, tau_lb=1.0, max_sweeps=10)
    args.update(kw)
    p = pkr.problem(**args)
    h = ctypes.c_void_p()
    return pkr._pkr.pkr_plan_create(ctypes.byref(p), None, ctypes.byref(h)), h


def test_invalid_problems_rejected_before_any_gpu_work(pkr):
    assert _create(pkr, order=7)[0] == -1                 # N=7 needs the 13-speed sets
    assert _create(pkr, tau_lb=0.5)[0] == -1              # tau must exceed 1/2
    assert _create(pkr, lattice="D2Q169", order=7)[0] == -1   # 2D set on a 3D grid
    assert _create(pkr, shape=(0, 8, 8))[0] == -1
    assert _create(pkr, max_sweeps=0)[0] == -1
    assert _create(pkr, precision="mixed_fx64")[0] == -1  # ladders: pkr_solve and contexts
    p = pkr.problem("D3Q111", (8, 8, 8), 5, tau_lb=1.0)
    p.tol_kind = 7
    h = ctypes.c_void_p()
    assert pkr._pkr.pkr_plan_create(ctypes.byref(p), None, ctypes.byref(h)) == -1


def test_stability_precheck(pkr):
    """tau_lb = 0.6 on the N=5 3D set has growing modes (the oracle's
    instability test shows them); the plan is refused with PKR_EUNSTABLE.
    D3Q19 with N=1 (positive weights) is accepted by the pre-check."""
    assert _create(pkr, tau_lb=0.6)[0] == -3
    assert _create(pkr, lattice="D2Q169", shape=(16, 16), order=7, tau_lb=0.7)[0] == -3
    rc, h = _create(pkr, lattice="D3Q19", order=1, tau_lb=0.6)
    assert rc in (0, -6)   # passes the pre-check; -6 where no GPU is present
    if rc == 0:
        pkr._pkr.pkr_plan_destroy(h)


def test_fixed_point_fft_validation(pkr):
    """The FFT comparator checks its problem on the host before any CUDA call."""
    rho = np.zeros((4, 4, 4))
    phi = np.zeros((4, 4, 4))

    def call(prob):
        st = pkr._pkr.pkr_stats()
        return pkr._pkr.pkr_fixed_point_fft(ctypes.byref(prob), rho.ctypes.data, phi.ctypes.data,
                                            1, ctypes.byref(st), None)
    assert call(pkr.problem("D3Q111", (4, 4, 4), 5, tau_lb=0.5)) == -1
    assert call(pkr.problem("D3Q111", (4, 4, 4), 5, tau_lb=0.6)) == -3
    assert call(pkr.problem("D3Q111", (4, 4, 4), 9, tau_lb=1.0)) == -1
    bad = pkr.problem("D3Q111", (4, 4, 4), 5, tau_lb=1.0)
    bad.dim = 2
    assert call(bad) == -1
    st = pkr._pkr.pkr_stats()
    assert pkr._pkr.pkr_fixed_point_fft(ctypes.byref(bad), None, None, 1, ctypes.byref(st),
                                        None) == -1
    assert not phi.any()


def test_plan_bytes(pkr):
    p = pkr.problem("D3Q111", (256, 256, 256), 5, tau_lb=1.0)
    b = ctypes.c_size_t()
    assert pkr._pkr.pkr_plan_bytes(ctypes.byref(p), ctypes.byref(b)) == 0
    V = 256 ** 3
    assert 2 * 111 * V * 8 < b.value < 2 * 111 * V * 8 + 3 * V * 8
    p32 = pkr.problem("D3Q111", (256, 256, 256), 5, tau_lb=1.0, precision="fp32")
    b32 = ctypes.c_size_t()
    assert pkr._pkr.pkr_plan_bytes(ctypes.byref(p32), ctypes.byref(b32)) == 0
    assert b32.value < 0.55 * b.value


def test_context_config_validation(pk_cfg=None):
    import paper_1504_05869_gb300 as pk
    pk._pkr.load()

    def create(**kw):
        cfg = pk.pkr_ctx_config()
        cfg.lattice, cfg.order, cfg.precision = pk.LATTICES["D3Q111"], 5, 1
        cfg.check_every, cfg.hbm_budget_bytes, cfg.variant = 8, 10 ** 9, -1
        for k, v in kw.items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        return pk._pkr.pkr_ctx_create(ctypes.byref(cfg), None, ctypes.byref(h))

    assert create(check_every=0) == -1
    assert create(hbm_budget_bytes=0) == -1
    assert create(precision=7) == -1
    assert create(precision=3) == -1      # binary16 storage: pkr_solve only
    assert create(precision=8) == -1
    assert create(variant=99) == -1
    # the plan sweep's warp-specialised variants have no batch form
    nb = pk._pkr.pkr_batch_variant_count(pk.LATTICES["D3Q111"])
    assert 0 < nb < pk._pkr.pkr_variant_count(pk.LATTICES["D3Q111"])
    assert create(variant=nb) == -1
    for name in ("D1Q5", "D3Q19"):
        assert pk._pkr.pkr_batch_variant_count(pk.LATTICES[name]) == \
            pk._pkr.pkr_variant_count(pk.LATTICES[name])
    assert pk._pkr.pkr_batch_variant_count(42) < 0
    assert create(order=7) == -1
    assert create(lattice=42) == -1


def test_site_count_limits_rejected_on_the_host(pkr):
    """The flat site index is 32-bit: V = 2^31 is refused (PKR_EINVAL) by
    every entry point before any device work; 2^31 - 1 passes validation
    (pkr_plan_bytes reports its size)."""
    big = (1024, 1024, 2048)                       # numpy order: V = 2^31
    assert _create(pkr, shape=big)[0] == -1
    p = pkr.problem("D3Q111", big, 5, tau_lb=1.0)
    b = ctypes.c_size_t()
    assert pkr._pkr.pkr_plan_bytes(ctypes.byref(p), ctypes.byref(b)) == -1
    st = pkr._pkr.pkr_stats()
    dummy = ctypes.c_void_p(16)                    # never dereferenced: refused first
    assert pkr._pkr.pkr_solve(ctypes.byref(p), dummy, dummy, 0, ctypes.byref(st), None) == -1
    assert pkr._pkr.pkr_fixed_point_fft(ctypes.byref(p), dummy, dummy, 0, ctypes.byref(st),
                                        None) == -1
    ok = pkr.problem("D1Q5", (2 ** 31 - 1,), 3, tau_lb=1.0)
    assert pkr._pkr.pkr_plan_bytes(ctypes.byref(ok), ctypes.byref(b)) == 0
    assert b.value > 2 * 5 * (2 ** 31 - 1) * 8
    out = (ctypes.c_double * 3)()
    for V in (0, -5, 2 ** 31):
        assert pkr._pkr.pkr_residual_noalloc(dummy, dummy, V, out, None) == -1


def test_null_handles_and_pointers_rejected(pkr):
    """Every entry point that takes a handle or an output pointer refuses NULL
    with PKR_EINVAL before any device work; destroying NULL is a no-op
    (PKR_OK); the handle queries return their empty values."""
    L = pkr._pkr
    st = L.pkr_stats()
    dummy = ctypes.c_void_p(16)                     # never dereferenced: refused first
    p = pkr.problem("D3Q111", (8, 8, 8), 5, tau_lb=1.0)
    assert L.pkr_plan_create(ctypes.byref(p), None, None) == -1
    assert L.pkr_plan_create(None, None, ctypes.byref(ctypes.c_void_p())) == -1
    assert L.pkr_plan_destroy(None) == 0
    assert L.pkr_plan_load_source(None, dummy, 0) == -1
    assert L.pkr_plan_run(None, 1, 0.0, 0, 1, ctypes.byref(st)) == -1
    assert L.pkr_plan_sweeps(None, 1) == -1
    assert L.pkr_plan_phi(None, dummy, 0) == -1
    assert L.pkr_plan_autotune(None, 1, None, None) == -1
    assert L.pkr_plan_import(None, None) == -1
    assert L.pkr_plan_steps(None) == 0
    assert L.pkr_plan_populations(None) is None
    assert L.pkr_solve(None, dummy, dummy, 0, ctypes.byref(st), None) == -1
    assert L.pkr_solve(ctypes.byref(p), None, dummy, 0, ctypes.byref(st), None) == -1
    assert L.pkr_solve(ctypes.byref(p), dummy, None, 0, ctypes.byref(st), None) == -1
    assert L.pkr_plan_bytes(ctypes.byref(p), None) == -1
    assert L.pkr_tau_from_knudsen(pkr.LATTICES["D3Q111"], 0.2, None, None) == -1
    out = (ctypes.c_double * 3)()
    assert L.pkr_residual_noalloc(None, dummy, 8, out, None) == -1
    assert L.pkr_residual_noalloc(dummy, dummy, 8, None, None) == -1
    cfg = pkr.pkr_ctx_config()
    assert L.pkr_ctx_create(None, None, ctypes.byref(ctypes.c_void_p())) == -1
    assert L.pkr_ctx_create(ctypes.byref(cfg), None, None) == -1
    ticket = ctypes.c_uint64()
    assert L.pkr_submit(None, ctypes.byref(p), dummy, dummy, 0, ctypes.byref(ticket)) == -1
    assert L.pkr_poll(None, 0, ctypes.byref(st)) == -1
    assert L.pkr_ctx_wait(None, 0, ctypes.byref(st)) == -1
    assert L.pkr_ctx_run(None, 1) == -1
    assert L.pkr_ctx_info(None, None, None, None, None, None) == -1
    assert L.pkr_ctx_release(None, 1) == -1
    assert L.pkr_ctx_destroy(None) == 0


def test_struct_layouts_match_the_header(pkr, tmp_path):
    """The ctypes mirrors of pkr_problem, pkr_stats and pkr_ctx_config have
    the C structs' field names, order, offsets and sizes: a C program built
    against include/pkr.h prints offsetof/sizeof of every field the binding
    declares, and the struct sizes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [pkr._pkr.pkr_problem, pkr._pkr.pkr_stats, pkr._pkr.pkr_ctx_config]
    lines = ['#include <stdio.h>', '#include "pkr.h"', "int main(void) {"]
    want = []
    for st in structs:
        name = st.__name__
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        want.append(ctypes.sizeof(st))
        for field, ftype in st._fields_:
            lines.append(f'printf("%zu %zu\\n", offsetof({name}, {field}), '
                         f'sizeof((({name} *)0)->{field}));')
            want.append((getattr(st, field).offset, ctypes.sizeof(ftype)))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = []
    for row in out:
        parts = row.split()
        if len(parts) == 1:
            got.append(int(parts[0]))
        elif len(parts) == 2:
            got.append((int(parts[0]), int(parts[1])))
    assert got == want


def test_enum_constants_match_the_header(pkr, tmp_path):
    """The binding's status, lattice, precision and tolerance-kind constants
    equal the header's enumerators (printed by a C program built against
    include/pkr.h)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    b = pkr._pkr
    names = [n for n in dir(b) if n.startswith("PKR_") and isinstance(getattr(b, n), int)]
    pairs = [(n, getattr(b, n)) for n in sorted(names)]
    pairs += [(f"PKR_{k}", v) for k, v in sorted(b.LATTICES.items())]
    assert len(pairs) > 20
    lines = ['#include <stdio.h>', '#include "pkr.h"', "int main(void) {"]
    lines += [f'printf("%d\\n", (int){n});' for n, _ in pairs]
    lines += ["return 0;", "}"]
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "enums")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [v for _, v in pairs], pairs
