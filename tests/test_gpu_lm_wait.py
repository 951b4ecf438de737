"""The LM kernel's bounded waits (Sec. 3.2.3 refinement runs on staged
tiles of the mode table): a wait made to run out marks the frame, the call
returns RL_ERR_TIMEOUT with no result, the GPU stays usable, and the next
call with the default bound matches the FP64 oracle.  Nothing faults or
hangs: the copies the kernel waited for still land, and it drains them
with the full bound before it exits."""
import pytest

from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_lm_wait_runs_out_then_recovers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_12163_gb300 as rg
    ctx = rg.Context(0, arena_bytes=2 << 30)
    w = H.WORKLOADS[H.SMALL]
    g = H.gpu_model(ctx, w)
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 1)
    d, c, T, seed = w.query(0)
    orun, _ = H.oracle_query(w.name, 0, w.ransac)
    assert orun.result["n_hypotheses"] > 0              # the query reaches LM
    rel.set_wait_limit(0)                               # every tile wait gives up at once
    with pytest.raises(rg.RelocError) as e:
        rel.relocalise(d, c, w.K, seed)
    assert e.value.status == 5                          # RL_ERR_TIMEOUT
    torch.cuda.synchronize()                            # the context is still usable
    rel.set_wait_limit(-1)
    for use_graphs in (False, True):
        rel.set_graphs(use_graphs)
        gr = rel.relocalise(d, c, w.K, seed)
        orun, _ = H.oracle_query(w.name, 0, w.ransac)
        H.compare_results(rg, gr, rel.debug(0), orun, w.ransac, f"after timeout, graphs={use_graphs}")
    rel.close()
    scene.close()
    g.close()
    ctx.close()
