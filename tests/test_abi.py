"""The C-ABI library loads on a machine without a GPU, exports every symbol that
include/bnb.h declares, and refuses work cleanly when no device is present."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_04551_b300 import build
    build.build()
    import paper_2602_04551_b300 as b
    return b


def _declared(header="bnb.h"):
    txt = open(os.path.join(ROOT, "include", header)).read()
    return set(re.findall(r"\b(bnb_[a-z_0-9]+)\s*\(", txt)) - {"bnb_handle"}


def _exported(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True, check=True).stdout
    return set(re.findall(r" T (bnb_[a-z_0-9]+)", out))


def test_header_symbols_exported(lib):
    exported = _exported(lib.LIB_PATH)
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, declared - exported
    assert set(lib.SYMBOLS) == declared


def test_diagnostics_library_exports_its_header_and_the_product_does_not(lib):
    """The diagnostics (include/bnb_diag.h) live in libbnb_diag.so: it exports every call
    the header declares, the product library exports none of them, and the diagnostics
    library loads with its prototypes (their argument counts match the header)."""
    declared = _declared("bnb_diag.h")
    assert declared == set(lib.DIAG_SYMBOLS)
    assert declared <= _exported(lib.DIAG_LIB_PATH)
    assert not (declared & _exported(lib.LIB_PATH))
    raw = lib.load_diag_library()
    arity = _header_arity("bnb_diag.h")
    assert set(arity) == declared
    for name, count in arity.items():
        assert len(getattr(raw, name).argtypes) == count, name
    if raw.bnb_diag_wait_expiry(0, 0.001, None, None) != lib.BNB_EINVAL:
        raise AssertionError("bad limits must be rejected before any device work")
    import ctypes
    us, nb, err = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    for bad in [(0, 3, 88, 8, 5), (120, 1, 88, 8, 5), (120, 3, 90, 8, 5), (120, 3, 88, 0, 5),
                (120, 3, 88, 8, 0), (120, 8, 256, 8, 5)]:   # the last needs 513 KB of ring
        rc = raw.bnb_diag_tma_stream(*bad, ctypes.byref(us), ctypes.byref(nb), ctypes.byref(err))
        assert rc == lib.BNB_EINVAL, (bad, rc)


def test_options_default_and_errors(lib):
    o = lib.bnb_options_default()
    assert o.M == 0.0 and o.rho == 1.0 and o.batch_K == 512 and o.node_tol == 1e-4
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present: the no-device error path is not reachable")
    with pytest.raises(lib.BnbError) as ei:
        lib.bnb_create(np.ones((4, 3)), np.ones(4), 0.1, 0.1, lib.bnb_options_default(M=1.0))
    assert ei.value.code in (lib.BNB_ENODEV, lib.BNB_EINVAL)


def test_struct_layouts_match_header(lib, tmp_path):
    """The ctypes mirrors of bnb_options, bnb_stats and bnb_progress have the size and
    the field offsets a C compiler gives the header's structs (a drifted binding would
    marshal garbage into the library)."""
    import ctypes
    structs = {"bnb_options": lib.bnb_options, "bnb_stats": lib.bnb_stats,
               "bnb_progress": lib.bnb_progress}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "bnb.h"', "int main(void) {"]
    for name, cls in structs.items():
        src.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            src.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = 0
    for line in out.splitlines():
        name, field, value = line.split()
        cls = structs[name]
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (name, field, got, value)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_options_reject_unknown_fields(lib):
    o = lib.bnb_options_default(M=2.0, fused_shape=4, u_shape=1)
    assert (o.M, o.fused_shape, o.u_shape) == (2.0, 4, 1)
    with pytest.raises(TypeError):
        lib.bnb_options_default(M=1.0, fused_shap=3)


def test_footprint_host_arithmetic(lib):
    """bnb_footprint (used to admit solves under an HBM budget) needs no device: it grows
    with every dimension, covers at least the resident data and node state, rejects bad
    sizes, and the largest serving request fits the serving loop's 150 GB budget."""
    def fp(n, p, **kw):
        return lib.bnb_footprint(n, p, lib.bnb_options_default(M=1.0, **kw))

    base = fp(1000, 5000, batch_K=512)
    assert fp(2000, 5000, batch_K=512) > base
    assert fp(1000, 10000, batch_K=512) > base
    assert fp(1000, 5000, batch_K=1024) > base
    assert fp(1000, 5000, batch_K=512, queue_capacity=1 << 22) > fp(1000, 5000, batch_K=512,
                                                                   queue_capacity=1 << 18)
    for n, p, K in [(200, 50, 64), (1000, 5000, 512), (5000, 50000, 2048)]:
        # X in FP32 plus beta and V in FP32 for every slot, at the least
        assert fp(n, p, batch_K=K) >= 4 * n * p + 8 * K * p
    serve = dict(batch_K=256, queue_capacity=1 << 18, warm_capacity=1 << 14)
    assert fp(5000, 20000, **serve) < 150 << 30
    for n, p in [(0, 10), (10, 0), (-1, 5)]:
        with pytest.raises(lib.BnbError) as ei:
            fp(n, p)
        assert ei.value.code == lib.BNB_EINVAL


def _header_arity(header="bnb.h"):
    """Parameter count of every function the header declares."""
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(bnb_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_header(lib):
    """Every ctypes prototype has as many arguments as the header's declaration (a
    missing or extra argument would shift every pointer after it)."""
    raw = lib.load_library()
    arity = _header_arity()
    assert set(arity) == set(lib.SYMBOLS)
    for name, count in arity.items():
        assert len(getattr(raw, name).argtypes) == count, name


def test_null_handle_and_bad_sizes_rejected_without_a_device(lib):
    """Argument errors are reported as BNB_EINVAL before any device work, with a message;
    the calls that take no status (stream, destroy) accept NULL."""
    raw = lib.load_library()
    calls = {
        "bnb_relax_batch": (None, 4) + (None,) * 3 + (10,) + (None,) * 7,
        "bnb_relax_batch_device": (None, 4) + (None,) * 3 + (10,) + (None,) * 7,
        "bnb_dual_bound": (None, 4, None, None, None),
        "bnb_upper_batch": (None, 4, None, None, None),
        "bnb_solve": (None, 1e-4) + (None,) * 5,
        "bnb_solve_start": (None, 1e-4),
        "bnb_solve_launch": (None, 1),
        "bnb_solve_poll": (None, None),
        "bnb_solve_finish": (None,) * 6,
        "bnb_root_heuristic": (None, None, None),
        "bnb_profile_round": (None, None, None, 15),
        "bnb_get_histograms": (None, None, 0, None, 0),
        "bnb_get_stats": (None, None),
        "bnb_get_node_log": (None, 0, None, None, None, None),
        "bnb_dual_bound_static": (None, None, 10, 20, 0.1, 0.01, 1.0, 4, None, None, None, None),
    }
    for name, args in calls.items():
        assert getattr(raw, name)(*args) == lib.BNB_EINVAL, name
    X, y = np.ones((4, 3)), np.ones(4)
    o = lib.bnb_options_default(M=1.0)
    import ctypes
    h = ctypes.c_void_p()
    for n, p in [(0, 3), (4, 0), (-2, 3)]:
        rc = raw.bnb_create(lib._ptr(X), lib._ptr(y), n, p, 0.1, 0.1, ctypes.byref(o), ctypes.byref(h))
        assert rc == lib.BNB_EINVAL
        assert b"positive" in raw.bnb_last_error(None)
    assert raw.bnb_create(None, lib._ptr(y), 4, 3, 0.1, 0.1, ctypes.byref(o), ctypes.byref(h)) \
        == lib.BNB_EINVAL
    assert raw.bnb_create_device(None, None, 4, 3, 0.1, 0.1, ctypes.byref(o), ctypes.byref(h)) \
        == lib.BNB_EINVAL
    assert raw.bnb_stream(None) is None
    raw.bnb_destroy(None)


def test_plain_c_program_links_and_calls_the_library(lib, tmp_path):
    """The boundary is a C ABI: a C program that includes only bnb.h links against
    libbnb.so and calls the entry points that need no device."""
    src = r'''
#include <stdio.h>
#include <string.h>
#include "bnb.h"
int main(void) {
  bnb_options o;
  if (bnb_options_default(&o) != 0) return 1;
  size_t bytes = 0;
  if (bnb_footprint(1000, 5000, &o, &bytes) != 0 || bytes == 0) return 2;
  if (bnb_footprint(0, 5000, &o, &bytes) != BNB_EINVAL) return 3;
  double X[6] = {1, 2, 3, 4, 5, 6}, y[3] = {1, 2, 3};
  bnb_handle* h = NULL;
  if (bnb_create(X, y, 0, 2, 0.1, 0.1, &o, &h) != BNB_EINVAL || h != NULL) return 4;
  if (strstr(bnb_last_error(NULL), "positive") == NULL) return 5;
  if (bnb_solve_launch(NULL, 1) != BNB_EINVAL) return 6;
  bnb_destroy(NULL);
  printf("ok %zu\n", bytes);
  return 0;
}
'''
    c = tmp_path / "abi.c"
    c.write_text(src)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c),
                    "-L", libdir, "-lbnb", "-Wl,-rpath," + libdir, "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith("ok ")


def _header_defines():
    txt = open(os.path.join(ROOT, "include", "bnb.h")).read()
    return {m.group(1): int(m.group(2)) for m in
            re.finditer(r"^#define (BNB_[A-Z0-9_]+) \(?(-?\d+)\)?", txt, flags=re.M)}


def test_constants_match_header(lib):
    """Error codes and precisions have the header's values in the binding; every status
    code the header defines has a name (BNB_STATUS_X -> "x")."""
    defs = _header_defines()
    assert len(defs) == 19        # OK, six error codes, five precisions, seven statuses
    for name, value in defs.items():
        if name.startswith("BNB_STATUS_"):
            assert lib.STATUS_NAMES[value] == name[len("BNB_STATUS_"):].lower(), name
        else:
            assert getattr(lib, name) == value, name


def test_documented_defaults(lib):
    """bnb_options_default sets the defaults the header documents."""
    o = lib.bnb_options_default()
    want = dict(M=0.0, rho=1.0, node_tol=1e-4, max_admm_iter=400, check_every=10, batch_K=512,
                precision=lib.BNB_PREC_TC3, use_graphs=1, time_limit_s=3600.0, max_nodes=10**9,
                queue_capacity=1 << 20, warm_capacity=0, support_max=200, ub_max_iter=200, device=0,
                stream=None, relax_alpha=1.0, root_heuristic=1, max_depth=256, lockstep=0,
                mv_crossover=-1, fused_shape=0, u_shape=0, ub_polish=1, fused_width=0, fused_select=0, exact_bounds=0, log_nodes=0,
                early_branch=0)
    assert {k for k, _ in o._fields_} == set(want)
    for k, v in want.items():
        assert getattr(o, k) == v, k


def test_option_validation_on_the_host(lib):
    """Every option rule of bnb_create is checked on the host before any device work:
    each bad value returns BNB_EINVAL with its message, and a valid set reaches the
    device check (BNB_ENODEV here).  The data pointers are placeholders that the library
    never dereferences before that check, so the test runs only without a device."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present: the placeholder pointers would reach the device")
    raw = lib.load_library()
    ph = ctypes.c_void_p(4096)          # placeholder device pointers, never dereferenced
    h = ctypes.c_void_p()

    def create(lam0=0.1, lam2=0.01, **kw):
        o = lib.bnb_options_default(**dict(dict(M=1.0), **kw))
        rc = raw.bnb_create_device(ph, ph, 100, 50, lam0, lam2, ctypes.byref(o), ctypes.byref(h))
        return rc, raw.bnb_last_error(None).decode()

    assert create()[0] == lib.BNB_ENODEV
    bad = [
        (dict(lam0=-1.0), "lambda0"), (dict(lam2=0.0), "lambda2"), (dict(M=0.0), "options.M"),
        (dict(rho=0.0), "rho"), (dict(batch_K=0), "batch_K"), (dict(batch_K=70000), "batch_K"),
        (dict(support_max=0), "support_max"), (dict(support_max=300), "support_max"),
        (dict(check_every=0), "check_every"), (dict(max_depth=4), "max_depth"),
        (dict(max_depth=5000), "max_depth"), (dict(mv_crossover=-2), "mv_crossover"),
        (dict(mv_crossover=33), "mv_crossover"), (dict(fused_shape=5), "fused_shape"),
        (dict(u_shape=4), "u_shape"), (dict(relax_alpha=0.5), "relax_alpha"),
        (dict(relax_alpha=2.0), "relax_alpha"), (dict(queue_capacity=10), "queue_capacity"),
        (dict(queue_capacity=(1 << 30) + 1), "queue_capacity"), (dict(precision=7), "precision"),
        (dict(ub_polish=2), "ub_polish"), (dict(log_nodes=-1), "log_nodes"),
        (dict(log_nodes=70000), "log_nodes"), (dict(fused_width=-1), "fused_width"),
        (dict(fused_width=300), "fused_width"), (dict(fused_select=2), "fused_select"),
        (dict(exact_bounds=2), "exact_bounds"), (dict(early_branch=2), "early_branch"),
    ]
    for kw, word in bad:
        rc, msg = create(**kw)
        assert rc == lib.BNB_EINVAL and word in msg, (kw, rc, msg)
        assert h.value is None


def test_static_dual_bound_argument_checks_on_the_host(lib):
    """bnb_dual_bound_static rejects bad sizes, parameters and requests beyond its fixed
    scratch before any device work (placeholder pointers, never dereferenced)."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present: covered by the GPU no-allocation tests")
    raw = lib.load_library()
    ph = ctypes.c_void_p(4096)
    f = raw.bnb_dual_bound_static
    ok = dict(n=100, p=50, lam0=0.1, lam2=0.01, M=1.0, K=4)

    def call(**kw):
        a = dict(ok, **kw)
        return f(ph, ph, a["n"], a["p"], a["lam0"], a["lam2"], a["M"], a["K"], ph, ph, ph, None)

    for kw in (dict(n=0), dict(p=-1), dict(K=0), dict(lam0=-0.1), dict(lam2=0.0), dict(M=0.0),
               dict(K=70000), dict(p=50000, K=6000)):  # grid limit; 6000 x 198 doubles > 2^20
        assert call(**kw) == lib.BNB_EINVAL, kw
    assert f(None, ph, 100, 50, 0.1, 0.01, 1.0, 4, ph, ph, ph, None) == lib.BNB_EINVAL
    assert call(p=50000, K=5000) == lib.BNB_ENODEV   # 5000 x 198 doubles fit: reaches the device
