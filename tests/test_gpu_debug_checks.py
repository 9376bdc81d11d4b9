"""The debug library (device-side index checks; gini_debug_checks in
include/gini_mds.h) on the GPU: its self-test of a planted store past the
checked bound, and the hot paths against the oracle with every gini_check
clean.  The library is built on demand (build(debug=True)) and loaded in a
child process with GINI_DEBUG=1, since a process loads one library.

The release library is checked on the CPU: it reports no checks and its
self-test entry point launches nothing.
"""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_release_library_has_no_checks():
    from paper_2605_25124_gb300 import _lib, build
    build.build()
    if _lib.DEBUG:
        pytest.skip("this process loaded the debug library")
    L = _lib.lib()
    assert L.gini_debug_checks() == 0
    # release: GINI_EINVAL before any launch (the pointer is never touched)
    assert L.gini_selftest_index_check(None, 0, None) == _lib.GINI_EINVAL
    assert L.gini_status_str(_lib.GINI_EINDEX).startswith(b"GINI_EINDEX")


@pytest.mark.gpu
def test_debug_library_checks_pass_on_every_hot_path():
    from paper_2605_25124_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, GINI_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_checks_run.py")], env=env,
                       capture_output=True, text=True, timeout=1800)
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert line, r.stdout[-2000:] + r.stderr[-2000:]
    res = json.loads(line[-1])
    print(json.dumps(res["cases"], indent=1))
    assert res["debug_library"] == lib
    assert r.returncode == 0 and res["ok"], res["cases"]
