"""The debug build's device bounds checks (build(debug=True), loaded with SWMD_DEBUG=1
in a child process): with a word id one past the end of K^T planted in the corpus
from the host, a query on the resident (column-split) path and on the fused
per-iteration path reports the failed check through its status (SWMD_EINVAL) and
the kernels read index 0 instead.  The planted id stays inside the workspace's K^T
allocation (sized for 128 query columns), so even an unchecked read would not leave
device memory the library owns.  Unplanted queries give the release build's bits.
The release build refuses the hook."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth
E, C, (qi, qw) = synth.make("tiny")
res = {}
for path, what in (("resident", "nz"), ("fused", "slices")):
    corpus = swmd.corpus_from_synth(E, C, path=path)
    ok = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    res[path] = ok.tolist()
    swmd.swmd_debug_plant(corpus, what, 0, corpus.info().V_used)
    try:
        swmd.swmd_query(corpus, qi, qw, 1.0, 15)
        res[path + "_planted"] = "no error"
    except swmd.SwmdError as e:
        res[path + "_planted"] = [e.code, str(e)]
    corpus.close()
print(json.dumps(res))
"""


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_06433_gb300 import build
    build.build()
    build.build(debug=True)


def test_debug_build_reports_planted_ids(cuda):
    env = dict(os.environ, SWMD_DEBUG="1")
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, env=env,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    res = json.loads(p.stdout.strip().splitlines()[-1])
    E, C, (qi, qw) = synth.make("tiny")
    for path in ("resident", "fused"):
        release = swmd.swmd_query(swmd.corpus_from_synth(E, C, path=path), qi, qw, 1.0, 15)
        np.testing.assert_array_equal(np.array(res[path]), release)
        code, msg = res[path + "_planted"]
        assert code == swmd.SWMD_EINVAL and "bounds check" in msg, res[path + "_planted"]


def test_release_build_refuses_the_hook(cuda):
    E, C, _ = synth.make("tiny")
    corpus = swmd.corpus_from_synth(E, C)
    with pytest.raises(swmd.SwmdError) as e:
        swmd.swmd_debug_plant(corpus, "nz", 0, 0)
    assert e.value.code == swmd.SWMD_EINVAL and "debug builds" in str(e.value)
