"""The autotuner's cache file is read back by a new process (host only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, %r)
from paper_2403_06937_gb300 import build
build.build()
import paper_2403_06937_gb300 as tc
print(json.dumps([tc.autotune_lookup(11, 'bf16x3'), tc.autotune_lookup(11, 'fp64'), tc.autotune_lookup(12, 'bf16x3')]))
"""


def test_cache_file_is_read_on_first_lookup(tmp_path):
    cache = tmp_path / "tune.jsonl"
    # arch 0: the key a process without a CUDA device looks up
    cache.write_text('{"arch": 0, "n": 11, "precision": 1, "f64_tile": 64, "tc_group": 16, "tc_stages": 3, '
                     '"tc_shape": 2, "ms": 1.0}\n'
                     '{"arch": 0, "n": 11, "precision": 0, "f64_tile": 64, "tc_group": 8, "tc_stages": 0, "ms": 2.0}\n'
                     'not json\n')
    env = dict(os.environ, TC_AUTOTUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", SCRIPT % ROOT], env=env, capture_output=True, text=True, check=True)
    a, b, c = json.loads(out.stdout.strip().splitlines()[-1])
    assert a == {"f64_tile": 64, "tc_group": 16, "tc_stages": 3, "tc_shape": 2}
    assert b["f64_tile"] == 64 and b["tc_shape"] == 0       # a line without a shape: automatic
    assert c["tc_group"] == 8 and c["tc_stages"] == 4 and c["tc_shape"] == 0   # untuned: the defaults


BATCH_SCRIPT = r"""
import json, sys
sys.path.insert(0, %r)
from paper_2403_06937_gb300 import build
build.build()
import paper_2403_06937_gb300 as tc
ns = [6, 12, 9, 12]
out = [tc.batch_autotune_lookup(ns, 'bf16x3'), tc.batch_autotune_lookup(list(reversed(ns)), 'bf16x3'),
       tc.batch_autotune_lookup(ns, 'tf32'), tc.batch_autotune_lookup([6, 12, 9], 'bf16x3')]
tc.batch_autotune_set([6, 9], 'tf32', 16, 'single')
out.append(tc.batch_autotune_lookup([9, 6], 'tf32'))
print(json.dumps(out))
"""


def _fnv(ns):
    h = 1469598103934665603
    for x in sorted(ns):
        h ^= x
        h = (h * 1099511628211) % (1 << 64)
    return h


def test_batch_cache_is_keyed_by_composition(tmp_path):
    """A batch entry of the cache applies to that multiset of n (any order) and
    precision only; tc_batch_autotune_set pins one in the process."""
    cache = tmp_path / "tune.jsonl"
    cache.write_text('{"arch": 0, "batch": "%016x", "precision": 1, "tc_group": 4, "tc_shape": 3, "ms": 1.0}\n'
                     % _fnv([6, 12, 9, 12]))
    env = dict(os.environ, TC_AUTOTUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", BATCH_SCRIPT % ROOT], env=env, capture_output=True, text=True,
                         check=True)
    a, b, c, d, e = json.loads(out.stdout.strip().splitlines()[-1])
    assert a == b == {"tc_group": 4, "tc_shape": 3}
    assert c is None and d is None
    assert e == {"tc_group": 16, "tc_shape": 1}
