"""The long BER runner's checkpoint: a run stopped after some frames and
started again with the same checkpoint file gives exactly the counts of one
uninterrupted run (frames and noise are numbered globally)."""
import json

import pytest

from paper_1609_01567_gb300 import ber
from paper_1609_01567_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01567_gb300 import build
    build.build()
    from paper_1609_01567_gb300 import ldpc as mod
    return mod


def last_line(capsys):
    return json.loads([x for x in capsys.readouterr().out.splitlines() if x.startswith("{")][-1])


def test_resumed_run_equals_uninterrupted_run(ldpc, tmp_path, capsys):
    ck = str(tmp_path / "ber.json")
    common = ["--code", "n1008", "--ebn0", "1.5", "--batch", "500", "--msg", "f32", "--max-iter", "30",
              "--checkpoint", ck, "--chunk-frames", "400"]
    ber.main(["--frames", "1000"] + common)  # "stopped" after 1000 frames
    first = last_line(capsys)
    state = json.load(open(ck))
    assert [v["next_frame"] for v in state.values()] == [1000]
    ber.main(["--frames", "2600"] + common)  # resumed: frames 1000 .. 2599
    resumed = last_line(capsys)
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    whole = ber.summary(ber.simulate(h, code, 1.5, 2600, batch=500, max_iter=30), code.n)
    for k in ("frames", "frame_errors", "bit_errors", "mean_iters"):
        assert resumed[k] == whole[k], (k, resumed[k], whole[k])
    assert first["frames"] == 1000 and resumed["frames"] == 2600
    ber.main(["--frames", "2600"] + common)  # nothing left to run: the stored counts
    assert last_line(capsys)["frame_errors"] == whole["frame_errors"]
