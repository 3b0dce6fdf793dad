"""The failure path of the bounded device waits, made to happen without a
fault: a sort pass's look-back waits on a tile that nobody processes, gives
up after its iteration limit, and the library reports HGRD_ETIMEOUT; the
context stays usable (a full check afterwards equals the oracle)."""
import time

import pytest

import oracle
import paper_2604_02106_b300 as hg
import workloads

pytestmark = pytest.mark.gpu


def test_lookback_wait_runs_out_and_the_context_stays_usable():
    t0 = time.perf_counter()
    rc = hg.debug_lookback_timeout()
    assert rc == -8, hg.lib().hgrd_last_error().decode()  # HGRD_ETIMEOUT
    assert time.perf_counter() - t0 < 60
    w = workloads.config1(0)
    g = hg.check(w.text, w.binding, cap=1 << 16, flags=hg.NO_SMALL)
    o = oracle.check(w.text, w.binding, cap=1 << 16)
    assert g.witnesses == o.witnesses and g.n_witness == o.n_witness
