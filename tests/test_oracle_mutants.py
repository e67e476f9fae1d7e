"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch each one.  This shows the pins constrain every step of the oracle: a
dropped term, a wrong bit order, a wrong index or a transposed operand.

Each mutant is a textual substitution applied to a temporary copy of
oracle/stego_oracle.c, compiled with gcc and loaded through ctypes.  None of
them writes outside its buffers.
"""
import inspect
import math
import os
import shutil

import pytest

import oracle
import oracle_pins as P

MUTANTS = [
    # stream1 embed
    ("lsb_first", "(s >> (7u - (uint32_t)(k % 8u)))", "(s >> ((uint32_t)(k % 8u)))", 1),
    ("header_little_endian", "(8u * (3u - (uint32_t)q))", "(8u * (uint32_t)q)", 1),
    ("header_counts_bytes", "(uint32_t)(8u * m)", "(uint32_t)(m)", 1),
    ("clear_two_bits", "out[k] = (uint8_t)((cover[k] & 0xFEu) | bit);",
     "out[k] = (uint8_t)((cover[k] & 0xFCu) | bit);", 1),
    ("no_copy_of_tail", "memcpy(out, cover, (size_t)C);\n\n    for (k = 0;",
     "(void)0;\n\n    for (k = 0;", 1),
    # stream1 extract
    ("extract_lsb_first", "<< (7 - b)", "<< b", 1),
    ("extract_base_31", "base = 32u;", "base = 31u;", 1),
    ("header_weight_reversed", "<< (31u - (uint32_t)k)", "<< ((uint32_t)k)", 1),
    ("header_no_byte_check", "if (nbits % 8u != 0u)", "if (0)", 1),
    ("cap_check_dropped", "if (len > cap)\n            return OR_E_MSG_TOO_SMALL;\n        base = 32u;",
     "base = 32u;", 1),
    # paper2 embed
    ("paper_transposed", "((uint64_t)r * W + L * (uint64_t)i + j) * Cch + plane;\n                uint8_t y = msg",
     "((uint64_t)r * W + 4u * j + (uint64_t)i) * Cch + plane;\n                uint8_t y = msg", 1),
    ("paper_shift_i", "y = (uint8_t)(y >> (2 * i));", "y = (uint8_t)(y >> i);", 1),
    ("paper_mask3", "default: return 0xC0u;", "default: return 0x80u;", 1),
    ("paper_clear_one_bit", "out[x] = (uint8_t)((cover[x] & 0xFCu) | y);",
     "out[x] = (uint8_t)((cover[x] & 0xFEu) | y);", 1),
    ("paper_no_offset", "        off += L;\n        rem -= L;\n    }\n    return OR_OK;\n}\n\n/* Section VII",
     "        off += 0;\n        rem -= L;\n    }\n    return OR_OK;\n}\n\n/* Section VII", 1),
    ("paper_plane_ignored", "* Cch + plane;\n                uint8_t y = msg",
     "* Cch + 0u;\n                uint8_t y = msg", 1),
    # paper2 extract
    ("paper_extract_mask1", "(st[x] & 0x03u)", "(st[x] & 0x01u)", 1),
    ("paper_extract_shift_i", "y = (uint8_t)(y << (2 * i));", "y = (uint8_t)(y << i);", 1),
    ("paper_extract_no_zero", "msg[off + j] = 0;", "(void)0;", 1),
    # streamk
    ("streamk_field_lsb_first", "uint32_t pos = k - 1u - (uint32_t)(b % k);\n        out[x]",
     "uint32_t pos = (uint32_t)(b % k);\n        out[x]", 1),
    ("streamk_extract_field_order", "uint32_t pos = k - 1u - (uint32_t)(b % k);\n    return",
     "uint32_t pos = (uint32_t)(b % k);\n    return", 1),
    ("streamk_plane_ignored", "return plane_only ? x * Cch + plane : x;",
     "return plane_only ? x * Cch : x;", 1),
    ("streamk_header_no_byte_check", "if (nbits % 8u != 0u)", "if (0)", 2),
    ("streamk_clear_whole_field", "out[x] = (uint8_t)((out[x] & ~(1u << pos)) | ((uint32_t)bit << pos));",
     "out[x] = (uint8_t)((out[x] & ~((1u << k) - 1u) & 0xFFu) | ((uint32_t)bit << pos) | (out[x] & ((1u << pos) - 1u)));", 1),
    # statistics
    ("changed_positive_only", "if (d != 0)", "if (d > 0)", 1),
    ("sse_abs", "s += (uint64_t)(d * d);", "s += (uint64_t)(d < 0 ? -d : d);", 1),
]


# Mistakes in the Section VIII PSNR formula (oracle.psnr, Python): each is a
# textual substitution in that function's source, compiled into a
# replacement bound to a handle on the real oracle library.
PSNR_MUTANTS = [
    ("psnr_peak_256", "255.0 * 255.0", "256.0 * 256.0"),
    ("psnr_peak_unsquared", "255.0 * 255.0 * n", "255.0 * n"),
    ("psnr_20_log", "10.0 * math.log10", "20.0 * math.log10"),
    ("psnr_sse_over_n_inverted", "255.0 * 255.0 * n / sse", "255.0 * 255.0 / n * sse"),
    ("psnr_mse_per_plane", "255.0 * 255.0 * n / sse", "255.0 * 255.0 * (n / 3.0) / sse"),
    ("psnr_natural_log", "math.log10(", "math.log("),
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def _first_failure(o):
    for name, fn in P.PINS:
        try:
            fn(o)
        except AssertionError:
            return name
    return None


def test_unmutated_passes_all(oracle_lib):
    assert _first_failure(oracle_lib) is None


def _replace_nth(src, find, repl, nth):
    """Replace the nth (1-based) occurrence of find."""
    at = -1
    for _ in range(nth):
        at = src.find(find, at + 1)
        assert at >= 0
    return src[:at] + repl + src[at + len(find):]


@pytest.mark.parametrize("mname,find,repl,nth", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(workdir, mname, find, repl, nth):
    """nth: which occurrence of `find` in the oracle source is mutated."""
    with open(os.path.join(os.path.dirname(oracle.__file__), "stego_oracle.c")) as f:
        src = f.read()
    assert src.count(find) >= nth, "mutation site not found: " + mname
    mdir = workdir / mname
    mdir.mkdir()
    path = mdir / "m.c"
    path.write_text(_replace_nth(src, find, repl, nth))
    lib = oracle.build(str(path), str(mdir / "libm.so"))
    o = oracle.Oracle(lib)
    caught = _first_failure(o)
    shutil.rmtree(mdir, ignore_errors=True)
    assert caught is not None, "no pin caught mutant " + mname


@pytest.mark.parametrize("mname,find,repl", PSNR_MUTANTS, ids=[m[0] for m in PSNR_MUTANTS])
def test_psnr_mutant_is_caught(oracle_lib, mname, find, repl):
    src = inspect.getsource(oracle.psnr)
    assert find in src, "mutation site not found: " + mname
    ns = {"math": math}
    exec(src.replace(find, repl, 1), ns)
    o = oracle.Oracle(oracle_lib.path)
    o.psnr = ns["psnr"]
    caught = None
    for name, fn in P.PINS:
        try:
            fn(o)
        except (AssertionError, ArithmeticError, ValueError):
            caught = name
            break
    assert caught is not None, "no pin caught mutant " + mname
