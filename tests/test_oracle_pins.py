"""The oracle against facts it does not define itself (CPU only).

Also plants mistakes in copies of the oracle (on the CPU) and checks that the
pins catch each one: a pin set that a dropped term, a wrong bound or a lost
negation slips through would not pin anything.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import datagen as dg
import oracle
from tests import oracle_pins as pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin, oracle_lib):
    assert pin(oracle_lib) == []


def test_threaded_variant_matches_single(oracle_lib):
    tab = dg.config1_table(200_000)
    ot = oracle.OTable.from_table(tab)
    tree = dg.config1_predicate(0)
    c1 = oracle.count(ot, tree, threads=1)
    c4 = oracle.count(ot, tree, threads=4)
    assert c1 == c4 and c1 > 0
    assert np.array_equal(oracle.select(ot, tree, threads=1), oracle.select(ot, tree, threads=3))
    sub = oracle.count(ot, tree, 1000, 150_001) + oracle.count(ot, tree, 0, 1000) + \
        oracle.count(ot, tree, 150_001, None)
    assert sub == c1


def test_pushdown_threshold_is_strict(oracle_lib):
    """Algorithm 1 Execute: throw iff count > maxSize (a count equal to maxSize is materialised)."""
    col = np.arange(100, dtype=np.int32)
    t = oracle.OTable([col], ["i32"], [None])
    tree = dg.p_cmp(0, "<", 10)
    st, n, cols, ids = oracle.pushdown(t, tree, [0], 10)
    assert st == "OK" and n == 10 and list(cols[0]) == list(range(10))
    st, n, cols, ids = oracle.pushdown(t, tree, [0], 9)
    assert st == "TOO_LARGE" and n == 10 and cols is None
    assert oracle.max_rows_for_ratio(100, 0.1) == 10
    assert oracle.max_rows_for_ratio(3, 1 / 3) == 1
    st, n, _, _ = oracle.pushdown(t, dg.P_FALSE, [0], oracle.max_rows_for_ratio(100, 0.0))
    assert st == "OK" and n == 0


def test_type_errors():
    col = np.arange(10, dtype=np.int32)
    t = oracle.OTable([col, col.astype(np.float32)], ["i32", "f32"], [None, None])
    with pytest.raises(TypeError):
        oracle.count(t, dg.p_cmp(1, "<", 0.1))           # not exactly a float32
    with pytest.raises(TypeError):
        oracle.count(t, dg.p_cmp(0, "<", 1.5))           # float constant on an int column
    with pytest.raises(TypeError):
        oracle.count(t, dg.p_like(0, "a"))               # LIKE on a non-dictionary column
    with pytest.raises(IndexError):
        oracle.count(t, dg.p_cmp(5, "<", 1))


MUTANTS = {
    "between_lo_exclusive": ("return nd->i0 <= v && v <= nd->i1;", "return nd->i0 < v && v <= nd->i1;"),
    "between_operands_swapped": ("return nd->f0 <= v && v <= nd->f1;", "return nd->f1 <= v && v <= nd->f0;"),
    "not_dropped": ("return !eval_node(nodes, nd->child[0], cols, row);",
                    "return eval_node(nodes, nd->child[0], cols, row);"),
    "or_as_and": ("if (eval_node(nodes, nd->child[i], cols, row)) return 1;\n        return 0;",
                  "if (!eval_node(nodes, nd->child[i], cols, row)) return 0;\n        return 1;"),
    "and_drops_last_term": ("for (int32_t i = 0; i < nd->n_child; i++)\n            if (!eval_node",
                            "for (int32_t i = 0; i + 1 < nd->n_child; i++)\n            if (!eval_node"),
    "lt_as_le": ("case O_LT: return v < k;\n    case O_LE: return v <= k;\n    case O_GT: return v > k;\n    case O_GE: return v >= k;\n    }\n    return 0;\n}\n\nstatic int cmp_flt",
                 "case O_LT: return v <= k;\n    case O_LE: return v <= k;\n    case O_GT: return v > k;\n    case O_GE: return v >= k;\n    }\n    return 0;\n}\n\nstatic int cmp_flt"),
    "float_ne_as_eq": ("case O_NE: return v != k;\n    case O_LT: return v < k;\n    case O_LE: return v <= k;\n    case O_GT: return v > k;\n    case O_GE: return v >= k;\n    }\n    return 0;\n}\n\n/* P(R",
                       "case O_NE: return v == k;\n    case O_LT: return v < k;\n    case O_LE: return v <= k;\n    case O_GT: return v > k;\n    case O_GE: return v >= k;\n    }\n    return 0;\n}\n\n/* P(R"),
    "like_prefix_short": ("return strncmp(c->dict[code], nd->prefix, m) == 0;",
                          "return strncmp(c->dict[code], nd->prefix, m ? m - 1 : 0) == 0;"),
    "like_code_zero_excluded": ("if (code < 0 || code >= c->n_dict) return 0;",
                                "if (code <= 0 || code >= c->n_dict) return 0;"),
    "in_first_value_only": ("if (v == nd->ivals[i]) return 1;", "if (v == nd->ivals[0]) return 1;"),
    "int64_truncated": ("if (c->type == T_I64) return ((const int64_t*)c->data)[row];",
                        "if (c->type == T_I64) return (int32_t)((const int64_t*)c->data)[row];"),
    "count_skips_last_row": ("for (int64_t i = row_begin; i < row_end; i++)\n        n +=",
                             "for (int64_t i = row_begin; i + 1 < row_end; i++)\n        n +="),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    (tmp_path / "m.c").write_text(src.replace(old, new))
    so = str(tmp_path / "m.so")
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", str(tmp_path / "m.c"), "-o", so])
    # a child process, so that a mutant that crashes cannot take the test session down
    code = ("import sys; import oracle; from tests import oracle_pins as p; "
            f"f = p.run_all(oracle.load({so!r})); print(len(f)); sys.exit(0 if f else 3)")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode != 3, f"no pin catches mutant {name}"
    assert r.returncode == 0, f"mutant {name} crashed instead of failing a pin: {r.stderr[-500:]}"
