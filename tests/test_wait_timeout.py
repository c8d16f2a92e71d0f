"""A bounded device wait that runs out: the cluster merge's CTAs of one rank
issue no bulk copy (the testing hook of sqs_state_set_wait_test), so their
mbarrier wait reaches its short poll limit.  The kernel records the error
and finishes; the next waiting call returns SQS_ERR_TIMEOUT, and after
sqs_state_reset the same state computes the step correctly.  No GPU fault
is involved: the failure is the absence of a host-issued copy."""
import time

import numpy as np
import pytest

import oracle
from paper_2503_15118_gb300 import workloads as W
from tests.helpers import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


@pytest.mark.parametrize("widths", [[16, 16, 16, 16], [20, 32, 32]])
def test_cluster_wait_runs_out_then_recovers(sqs, widths):
    target = (1, 6)
    lo, hi, amps = W.random_state(widths, 50000, seed=31, pair_fraction=0.5, target=target)
    st = sqs.State(widths, eps=1e-14, merge=sqs.MERGE_CLUSTER)
    st.import_(lo, hi, amps)
    st.sync()
    assert st.lib.sqs_state_set_wait_test(st.h, 64, 0) == sqs.OK
    t0 = time.perf_counter()
    st.h_gate(*target)
    with pytest.raises(sqs.SqsError) as err:
        st.sync()
    assert err.value.status == sqs.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # Still refused until reset.
    with pytest.raises(sqs.SqsError):
        st.h_gate(*target)
        st.sync()
    assert st.lib.sqs_state_set_wait_test(st.h, 0, -1) == sqs.OK
    st.reset()
    st.import_(lo, hi, amps)
    st.h_gate(*target)
    assert st.stats()["steps_cluster"] >= 1
    o = oracle.OracleState(widths, eps=1e-14)
    o.import_(lo, hi, amps)
    o.h_gate(*target)
    assert compare_states(st.to_dict(), o.to_dict()) >= 1 - 1e-10
    st.close()


def test_wait_test_hook_rejects_bad_rank(sqs):
    st = sqs.State([8], eps=1e-14)
    assert st.lib.sqs_state_set_wait_test(st.h, 10, 8) == sqs.ERR_ARG
    assert st.lib.sqs_state_set_wait_test(st.h, 10, -1) == sqs.OK
    st.close()
