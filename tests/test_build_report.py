"""Register and spill budgets of the hot kernels, read from the ``-Xptxas -v``
report that the build writes (CPU only; skipped when the library has not been
built in this tree).

The measured rates depend on launch bounds that only pay while the bodies fit
them without spilling: 4 CTAs of 128 threads per SM (128 registers) for the
two-column step kernels, 6 (80 registers) for the one-column FP32 step kernel
and the one-column batch work list.  Held to fewer registers, the two-column
FP32 body spilled and lost 38 % of its rate, so a change that makes any of
these spill should be seen before it reaches a GPU.
"""
import os
import re

import pytest

from paper_1204_4098_gb300 import build

ENTRY = re.compile(
    r"Compiling entry function '([^']+)' for 'sm_103a'\n"
    r"(?:ptxas info\s*: Function properties for [^\n]*\n)?"
    r"\s*(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads\n"
    r"ptxas info\s*: Used (\d+) registers")


@pytest.fixture(scope="module")
def kernels():
    if not os.path.exists(build.REPORT):
        pytest.skip("no build report in this tree (build the library first)")
    text = open(build.REPORT).read()
    out = {}
    for name, _stack, spill_st, spill_ld, regs in ENTRY.findall(text):
        out[name] = (int(regs), int(spill_st), int(spill_ld))
    assert out, "the build report lists no kernels"
    return out


def pick(kernels, fragment):
    found = {k: v for k, v in kernels.items() if fragment in k}
    assert found, f"no kernel matching {fragment!r} in the build report"
    return found


# (mangled-name fragment, register limit, spill-store limit in bytes)
BUDGETS = [
    ("strip2_kernelINS_8StoreF32E", 128, 0),   # two columns per lane, FP32
    ("strip2_kernelINS_9StoreBF16E", 128, 0),  # two columns, BF16 deviations
    ("strip2_kernelINS_8StoreF16E", 128, 0),   # two columns, FP16 deviations
    ("strip_kernelINS_8StoreF32E", 80, 0),     # one column per lane, FP32
    ("batch_worklist_kernelILb0E", 80, 8),     # batch, one column (6 CTAs per SM): 4 B
    ("batch_worklist_kernelILb1E", 128, 16),   # batch, two columns: 8 B measured (76 B
                                               # before the item prologue's rows were
                                               # fetched together)
]


@pytest.mark.parametrize("fragment,max_regs,max_spill", BUDGETS,
                         ids=[b[0] for b in BUDGETS])
def test_hot_kernels_fit_their_launch_bounds(kernels, fragment, max_regs, max_spill):
    for name, (regs, spill_st, spill_ld) in pick(kernels, fragment).items():
        assert regs <= max_regs, (name, regs)
        assert spill_st <= max_spill and spill_ld <= max_spill + 8, (name, spill_st, spill_ld)
