"""Host logic of bench.py that needs no GPU: the source hash that decides whether the
committed ncu DRAM counters still describe the kernel being timed."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_comment_edits_keep_the_code_text_and_code_edits_change_it():
    b = _bench()
    src = "int f(int x)   // scale\n{\n    // twice\n    return 2 * x;\n}\n"
    commented = "// new header line\nint f(int x)   // scale by two\n{\n\n    return 2 * x;   // doubled\n}\n"
    changed = "int f(int x)   // scale\n{\n    return 3 * x;\n}\n"
    assert b.code_text(src) == b.code_text(commented)
    assert b.code_text(src) != b.code_text(changed)


def test_traffic_record_is_well_formed():
    # a record whose hash no longer matches is legitimate (the bench then reports null
    # traffic until the next capture); its fields must still be usable
    import json
    b = _bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name, r in rec.items():
        assert r["bytes_per_field"] > 0, name
        assert len(r["src_hash"]) == 16 and r["sources"], name
        b.src_hash(r["sources"])   # every listed source exists and hashes


def test_roofline_bytes_follow_the_staged_fp32_rule():
    """Algorithmic bytes of a pass: 4 B in + 4 B out per grid element and pair field, plus
    f(Lambda) (8 B per point) once per launch for the pass that scales; the apply roofline
    counts 16 N B per unique pair plus the compulsory FP64 input and output."""
    b = _bench()

    class S:
        n = (48, 48, 48)
        N = 48 ** 3
        n_orb = 128
        n_occ = 128

        def unique_pairs(self):
            return 8256

    s = S()
    r = b.roofline(s, "bf16x7", "pass3", 10.0, 10, 1, {"hbm_gbs": 6000.0})
    fields = 8256 / 10
    assert r["algorithmic_bytes_per_launch"] == 8 * s.N * fields + 8 * s.N
    assert abs(r["achieved"] - r["algorithmic_bytes_per_launch"] / 1e-3 / 1e9) < 1e-6
    assert r["kernel"].startswith("zpass_kernel")
    ra = b.roofline_apply(s, "bf16x7", 10.0, {"hbm_gbs": 6000.0})
    assert ra["bytes_per_apply"] == 16 * s.N * 8256 + 8 * s.N * 256


def test_tensor_roofline_counts_the_digit_products():
    """Algorithmic flops of the six mode products, 4 N (n1 + n2 + n3) per unique pair; the
    executed tensor flops multiply them by the digit products of one mode product (BF16X7: 7)
    and divide by the measured sustained bf16 rate (TF32X3: half of it)."""
    b = _bench()

    class S:
        n = (72, 72, 144)
        N = 72 * 72 * 144

        def unique_pairs(self):
            return 499600

    s = S()
    algo = 4.0 * s.N * (72 + 72 + 144) * 499600
    r = b.tensor_roofline(s, "bf16x7", 1000.0, {"bf16_tflops_sustained": 1700.0})
    assert abs(r["algorithmic_tflops"] - algo / 1e12) < 1e-9
    assert abs(r["executed_tflops"] - 7 * algo / 1e12) < 1e-9
    assert abs(r["frac"] - 7 * algo / 1e12 / 1700.0) < 1e-12
    rt = b.tensor_roofline(s, "tf32x3", 1000.0, {"bf16_tflops_sustained": 1700.0})
    assert rt["peak"] == 850.0 and rt["digit_products"] == 3
    assert "executed_tflops" not in b.tensor_roofline(s, "fp64", 1000.0, {})
