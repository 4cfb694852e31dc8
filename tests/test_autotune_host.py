"""Host logic of the autotuner: one tuning per (grid, order, precision,
layout) key, the choice pinned for every later request of the key (in memory
and across processes through the JSON file), and one tuning when several
threads ask for a new key at once. The GPU timing itself (`_tune`) is
replaced by a stand-in that records its calls; the GPU test
`test_autotuner_pins_one_choice_per_shape` runs the real one."""
import json
import threading
import time

from paper_1801_06364_b300.autotune import Autotuner, key_of


class CountingTuner(Autotuner):
    def __init__(self, *a, delay=0.0, **k):
        super().__init__(*a, **k)
        self.calls = []
        self.delay = delay

    def _tune(self, shape, N, precision, real, dx, c, pml_cells, pml_mu0, pml_mu1, stream):
        self.calls.append((tuple(shape), N, precision, real))
        time.sleep(self.delay)
        return {"schedule": "plane" if N < 5 else "split", "graph_steps": 4 * (len(self.calls)),
                "ms_per_step": 1.0, "candidates_ms_per_step": {}}


def test_key_names_grid_order_precision_and_layout():
    assert key_of((64, 96, 128), 5, "fp32", True) == "128x96x64/N5/fp32/real"
    assert key_of((32, 32, 32), 3, "fp64", False) == "32x32x32/N3/fp64/full"


def test_one_tuning_per_key_and_the_choice_is_pinned():
    t = CountingTuner()
    a = t.choice((64, 64, 64), 3)
    assert t.choice((64, 64, 64), 3) is a                 # pinned, not re-tuned
    b = t.choice((64, 64, 64), 5)                         # another order: its own tuning
    c = t.choice((64, 64, 64), 3, real_radiance=False)    # another layout: its own tuning
    assert len(t.calls) == 3
    assert a["graph_steps"] != b["graph_steps"] != c["graph_steps"]
    assert t.choice((64, 64, 64), 5) is b and len(t.calls) == 3


def test_choices_persist_through_the_file(tmp_path):
    path = str(tmp_path / "tune.json")
    t = CountingTuner(path)
    first = t.choice((96, 96, 96), 7)
    with open(path) as f:
        assert json.load(f)[key_of((96, 96, 96), 7, "fp32", True)] == first
    again = CountingTuner(path)                           # a later process
    assert again.choice((96, 96, 96), 7) == first
    assert again.calls == []


def test_concurrent_requests_for_a_new_key_tune_once():
    t = CountingTuner(delay=0.05)
    got = []
    threads = [threading.Thread(target=lambda: got.append(t.choice((128, 128, 128), 7))) for _ in range(8)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert len(t.calls) == 1
    assert all(g is got[0] for g in got)
