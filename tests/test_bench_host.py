"""Host-side pieces of bench.py: the committed ncu traffic belongs to the
current source of its kernel (else the bench reports traffic null), and the
autotune summary counts every choice."""
import bench


def test_committed_traffic_matches_kernel_source():
    t = bench.NCU_TRAFFIC
    assert t["bytes_per_launch"] > 0
    assert bench._kernel_sha(t["kernel"]) == t["source_sha"], \
        "the Schur kernel changed since its DRAM traffic was captured: capture it again"


def test_tune_summary_counts_choices():
    class Fake:
        def h2_info(self):
            return {"levels": 3}

        def h2_autotune_choice(self, level):
            return (32, 128, 256)[level], level % 2

    assert bench._tune_summary([Fake(), Fake()]) == "2/2/2 of 6, 2/6"
