"""Per-context device-memory accounting and the HBM budget (cc_lr_init's hbm_budget_bytes).

Every allocation a context makes, at init or in any later call, is charged to it and checked
against its budget before it is made; a call that would exceed the budget returns CCLR_ENOMEM.
"""
import pytest

from paper_2604_12914_gb300 import binding
from paper_2604_12914_gb300.inputs import make_config, random_amplitudes

pytestmark = pytest.mark.gpu


def _ctx(s, budget=0, prec="tf32"):
    return binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec=prec, hbm_budget=budget)


def test_budget_covers_allocations_after_init():
    s = make_config("C1")
    x1, x2 = random_amplitudes(s.o, s.v, seed=3)
    ref = _ctx(s)
    used0, peak0, budget0 = ref.cc_lr_memory()
    assert budget0 == 0 and 0 < used0 <= peak0
    ref.cc_lr_sigma(x1, x2)
    used1, peak1, _ = ref.cc_lr_memory()
    assert used1 > used0 and peak1 >= used1       # the first sigma allocates workspace
    ref.close()
    # a budget that init fits in, but not the first product's workspace
    ctx = _ctx(s, budget=peak0 + 4096)
    with pytest.raises(binding.CclrError) as e:
        ctx.cc_lr_sigma(x1, x2)
    assert e.value.status == binding.CCLR_ENOMEM
    assert "budget" in str(e.value)
    used, peak, budget = ctx.cc_lr_memory()
    assert budget == peak0 + 4096 and peak <= budget and used <= budget
    ctx.close()
    # and a budget that covers it all gives the same sigma as no budget
    ctx = _ctx(s, budget=peak1 + (64 << 20))
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    used, peak, budget = ctx.cc_lr_memory()
    assert peak <= budget
    ctx.close()


def test_budget_below_init_needs_fails_at_init():
    s = make_config("C1")
    with pytest.raises(binding.CclrError) as e:
        _ctx(s, budget=1 << 20)
    assert e.value.status == binding.CCLR_ENOMEM
