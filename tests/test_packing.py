"""Host-side packing arithmetic of the batching layer (no GPU)."""
from paper_2511_00737_gb300 import batching as BT
from paper_2511_00737_gb300 import workload as WL


def test_packed_offsets_and_groups():
    pb = BT.PackedBatch([5, 0, 300, 17], cap=256)
    assert pb.offsets == [0, 5, 5, 305]
    assert pb.total == 322 and pb.groups == 2
    assert pb.rows(2) == slice(5, 305)
    assert BT.PackedBatch([256], 256).groups == 1
    assert BT.PackedBatch([257], 256).groups == 2
    assert BT.PackedBatch([0], 256).groups == 1


def test_client_batch_sizes_are_log_uniform_and_bounded():
    b = WL.client_batches(2511, clients=64)
    assert len(b) == 64 and b.min() >= 1 and b.max() <= 4096
    w = WL.config("clients64")
    assert w.B == sum(w.clients) and len(w.clients) == 64


def test_arrivals_are_poisson_with_bounded_lognormal_sizes():
    t, s = WL.arrivals(1, 20000, rate_per_s=2000.0)
    assert abs(len(t) / t[-1] - 2000.0) / 2000.0 < 0.05
    assert s.min() >= 1 and s.max() <= 8192
    assert 25 <= sorted(s)[len(s) // 2] <= 40  # median ~ 32
