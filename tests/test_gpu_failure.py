"""Failure detection without a GPU fault: the bounded device wait the bulk-copy text path uses runs
out on an mbarrier that nothing arrives on, reports E_TIMEOUT through a status word the host reads,
and leaves the context usable; with the phase completed it returns at once."""
import pytest

import textgen
from oracle.recognizer import SerialRecognizer

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_bounded_wait_times_out_and_context_survives():
    assert lib.ridfa_check_bounded_wait(4096, True) == 0
    assert lib.ridfa_check_bounded_wait(4096, False) == -7
    assert lib.ridfa_check_bounded_wait(0, True) == -7          # no poll at all: out at once
    x = textgen.c1_text(20_000, seed=5)
    prog = lib.ridfa_compile(textgen.C1_RE)
    d = torch.from_numpy(x.copy()).to("cuda:0")
    assert lib.ridfa_recognize(prog, d, x.size, 8) == SerialRecognizer(textgen.C1_RE).accepts(x)
    assert lib.ridfa_last_status(prog) == 0
