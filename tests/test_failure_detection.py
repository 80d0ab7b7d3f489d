"""Failure detection on the device without a GPU fault: a bounded wait on a flag that nothing
sets gives up, the host reads COFFEE_ERR_TIMEOUT from the error word, and the context stays
usable (an assembly right after it is correct and reports no error)."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import HELMHOLTZ, TET, rel_err_per_cell

COFFEE_ERR_TIMEOUT = -6


@pytest.mark.gpu
def test_bounded_wait_gives_up_and_the_context_stays_usable():
    coffee.check_errors()  # start from a clean error word
    t0 = time.time()
    coffee.diag_wait_timeout()
    with pytest.raises(coffee.CoffeeError) as info:
        coffee.check_errors()
    waited = time.time() - t0
    assert info.value.status == COFFEE_ERR_TIMEOUT
    assert 0.3 < waited < 60.0, waited
    coffee.check_errors()  # the word was cleared
    mesh = meshgen.tet_mesh(4, perturb=0.15, seed=3)
    x = torch.from_numpy(mesh.coords).cuda()
    c2v = torch.from_numpy(mesh.cell2vert).cuda()
    out = coffee.assemble(HELMHOLTZ, 2, TET, x, c2v, precision=coffee.TF32X3)
    coffee.check_errors()
    ref = oracle.assemble(HELMHOLTZ, 2, TET, mesh.coords, mesh.cell2vert)
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5
