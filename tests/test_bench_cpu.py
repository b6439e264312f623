"""Host-side logic of bench.py that needs no GPU: the algorithmic byte counts
the roofline divides by, the exact-count test of the end-to-end upload and the
source hash that dates the committed ncu traffic."""
import importlib.util
import json
import os
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_of_the_dm256_cycle(bench):
    """DM at 4000 x 256^2, object 2048^2, one mode: Psi read, Psi' written and
    read again (24 B/px), I (4 B/px), O and P read + written (16 B/px)."""
    s = types.SimpleNamespace(N=256, K=1, J=4000, Ho=2048, Wo=2048)
    px = 256 * 256
    want = 4000 * px * 24 + 4000 * px * 4 + 2048 * 2048 * 16 + px * 16
    assert bench.alg_bytes_per_cycle(s, "DM") == want == 7408189440
    # AP never reads an old Psi
    assert bench.alg_bytes_per_cycle(s, "AP") == want - 4000 * px * 8


def test_kernel_models_per_frame(bench):
    s = types.SimpleNamespace(N=256, K=1, J=1, Ho=256, Wo=256)
    m = bench.kernel_models(s)
    assert m["col"]["bytes"] == 256 * 256 * 4          # the intensities
    assert m["row_fwd"]["bytes"] == 256 * 256 * 8      # Psi
    assert m["row_bwd"]["bytes"] == 256 * 256 * 8      # Psi'
    # two column transforms of 5 N log2 N flops per line, plus the per-pixel work
    assert m["col"]["flops"] == 2 * 5.0 * 256 * 256 * 8 + 42.0 * 256 * 256


def test_exact_counts(bench):
    x = np.array([[0.0, 1.0], [65535.0, 17.0]], dtype=np.float32)
    c = bench.exact_counts(x)
    assert c.dtype == np.uint16 and np.array_equal(c.astype(np.float32), x)
    assert bench.exact_counts(np.array([0.5], np.float32)) is None
    assert bench.exact_counts(np.array([65536.0], np.float32)) is None
    assert bench.exact_counts(np.array([-1.0], np.float32)) is None


def test_source_hash_dates_the_traffic_file(bench):
    h = bench.source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    # every entry names the sources it was taken on; the bench reports it only on a match
    for k in ("col", "row_fwd", "row_bwd", "obj_gather"):
        assert len(d[k]["source_hash"]) == 16
    assert (bench.ncu_traffic("col") is None) == (d["col"]["source_hash"] != h)


def test_code_hash_ignores_comments_only(bench):
    a = 'int f(int x) {  // twice\n    return 2 * x; /* the double */\n}\nconst char* s = "// kept";\n'
    b = 'int f(int x) {\n\n    return 2 * x;\n}\nconst char* s = "// kept";\n'
    c = 'int f(int x) {\n    return 3 * x;\n}\nconst char* s = "// kept";\n'
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
    assert '"// kept"' in bench._code_only(a)


def test_end_to_end_upload_form(bench):
    """The end-to-end leg's upload form: exact counts with few values >= 255
    go up in the one-byte form, exact counts with many large values as uint16,
    anything else as float32; an explicit choice is honoured or refused."""
    rng = np.random.default_rng(5)
    low = rng.poisson(3.0, size=(8, 16, 16)).astype(np.float32)
    low[0, 0, :5] = 300.0                                   # 5 of 2048 escapes
    high = rng.integers(200, 60000, size=(8, 16, 16)).astype(np.float32)
    frac = low.copy()
    frac[1, 2, 3] = 0.5
    args = lambda d: types.SimpleNamespace(e2e_dtype=d)
    scan = lambda x: types.SimpleNamespace(iobs=x)
    assert bench.e2e_form(args("auto"), scan(low)) == "u8"
    assert bench.e2e_form(args("auto"), scan(high)) == "u16"
    assert bench.e2e_form(args("auto"), scan(frac)) == "f32"
    assert bench.e2e_form(args("u16"), scan(low)) == "u16"
    assert bench.e2e_form(args("u8"), scan(high)) == "u8"
    assert bench.e2e_form(args("f32"), scan(low)) == "f32"
    with pytest.raises(SystemExit):
        bench.e2e_form(args("u8"), scan(frac))
