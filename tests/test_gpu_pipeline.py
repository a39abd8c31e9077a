"""Host-resident steps with overlapped copies (pipeline.pipelined_steps) give
the same bits as copying in, stepping and copying out one step at a time."""
import numpy as np
import pytest

from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_pipelined_steps_equal_serial_steps(prec):
    import torch

    import paper_1712_01294_gb300 as m
    from paper_1712_01294_gb300 import pipeline
    states = [cast_state(I.turbulence(14, seed=s), prec) for s in (1, 2, 3, 4, 5)]
    host_in = []
    for q in states:
        d = m.to_device(q, prec)
        host_in.append({k: v.cpu().pin_memory() for k, v in d.items()})
    stream = torch.cuda.Stream()
    ctx = m.Context([states[0].N], m.default_params(precision=prec), stream=stream)
    serial = []
    with torch.cuda.stream(stream):
        for h in host_in:
            d = {k: v.cuda() for k, v in h.items()}
            ctx.step(d)
            serial.append({k: d[k].cpu() for k in pipeline.OUT_FIELDS})
        torch.cuda.synchronize()
        host_out = [{k: torch.empty_like(h[k]).pin_memory() for k in pipeline.OUT_FIELDS} for h in host_in]
        pipeline.pipelined_steps(ctx, host_in, host_out)
        torch.cuda.synchronize()
    assert ctx.status(reset=True)["ok"]
    for a, b in zip(serial, host_out):
        for k in pipeline.OUT_FIELDS:
            assert torch.equal(a[k], b[k]), k
