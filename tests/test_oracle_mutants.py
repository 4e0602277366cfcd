"""Plant plausible mistakes in a copy of the oracle (CPU only) and check
that the independent pins catch every one of them."""
import os
import shutil

import pytest

import oracle
from tests import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = [
    ("predicate drops the other-level term",
     "if (L[u] != L[w] || (L[u] == L[w] && v < w)) ++c;", "if (L[u] == L[w] && v < w) ++c;"),
    ("predicate compares w with u instead of v",
     "if (L[u] != L[w] || (L[u] == L[w] && v < w)) ++c;",
     "if (L[u] != L[w] || (L[u] == L[w] && u < w)) ++c;"),
    ("predicate direction reversed",
     "if (L[u] != L[w] || (L[u] == L[w] && v < w)) ++c;",
     "if (L[u] != L[w] || (L[u] == L[w] && w < v)) ++c;"),
    ("count visits both directions of a cover edge",
     "if (L[u] == L[v] && u < v) T += cover_edge_count(off, cols, L, u, v);\n    }\n  }\n  return T;\n}\n\n/* Per-edge counts",
     "if (L[u] == L[v]) T += cover_edge_count(off, cols, L, u, v);\n    }\n  }\n  return T;\n}\n\n/* Per-edge counts"),
    ("level not incremented", "L[y] = L[x] + 1;", "L[y] = L[x];"),
    ("root tie-break picks the highest id",
     "if (off[v + 1] - off[v] > off[r0 + 1] - off[r0]) r0 = v;",
     "if (off[v + 1] - off[v] >= off[r0 + 1] - off[r0]) r0 = v;"),
    ("first root is the lowest id, not the max degree",
     "if (off[v + 1] - off[v] > off[r0 + 1] - off[r0]) r0 = v;", ";"),
    ("unvisited components never restarted",
     "if (L[v] == OR_UNVISITED) bfs_from(v, off, cols, L, queue);", ";"),
    ("cover set keeps both orientations",
     "if (u < v && L[u] == L[v]) {\n        if (uv && h < cap)",
     "if (u != v && L[u] == L[v]) {\n        if (uv && h < cap)"),
    ("cover set keeps level-crossing edges",
     "if (u < v && L[u] == L[v]) {\n        if (uv && h < cap)", "if (u < v) {\n        if (uv && h < cap)"),
    ("plain apex cut against u", "else { if (a > v) ++c; ++i; ++j; }",
     "else { if (a > u) ++c; ++i; ++j; }"),
    ("all-core cover loop keeps both orientations",
     "if (L[u] == L[v] && u < v) T += cover_edge_count(off, cols, L, u, v);\n    }\n  }\n  return T;\n}\n\nOR_EXPORT uint64_t or_plain_count_mt",
     "if (L[u] == L[v]) T += cover_edge_count(off, cols, L, u, v);\n    }\n  }\n  return T;\n}\n\nOR_EXPORT uint64_t or_plain_count_mt"),
    ("all-core plain loop takes u > v too",
     "      if (u < v) T += plain_edge_count(off, cols, u, v);\n    }\n  }\n  return T;\n}\n\n/* Per-edge",
     "      if (u != v) T += plain_edge_count(off, cols, u, v);\n    }\n  }\n  return T;\n}\n\n/* Per-edge"),
    ("all-edge counts skip the level test",
     "if (u < v && L[u] == L[v]) {\n        if (h < cap)", "if (u < v) {\n        if (h < cap)"),
    ("enumerator apex cut dropped", "if (x > b) {", "if (x != b) {"),
    ("merge advances the wrong list", "if (a < b) {\n      ++i;", "if (a < b) {\n      ++j;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    mut = src.replace(old, new)
    p = tmp_path / "oracle_mut.c"
    p.write_text(mut)
    lib = oracle.compile_source(str(p), str(tmp_path / "liboracle_mut.so"))
    orc = oracle.Oracle(lib)
    failures = []
    for check in (pins.check_closed_forms, pins.check_brute_force, pins.check_trace,
                  pins.check_root_invariance):
        try:
            failures += check(orc)
        except Exception as e:  # a mutant may also crash a check
            failures.append(repr(e))
        if failures:
            break
    assert failures, f"mutant '{name}' passed every pin"
