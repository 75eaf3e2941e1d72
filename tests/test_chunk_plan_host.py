"""The split search behind the small-omega chunk table (no GPU): with equal
throughput for every omega count a request stays one chunk; when a 1- and a
32-omega chunk are much faster than a 33-omega one, 33 omegas split as 1 + 32,
and the per-chunk charge keeps near-ties in one chunk."""
from paper_1609_08146_gb300.tune_chunks import first_chunks


def test_uniform_throughput_keeps_one_chunk():
    first = first_chunks({n: 1.0 for n in range(1, 65)})
    assert first[1:] == list(range(1, 65))


def test_fast_classes_are_split_out():
    rate = {n: 1.0 for n in range(1, 65)}
    rate[1] = rate[32] = 10.0
    first = first_chunks(rate)
    assert first[33] == 1 and first[32] == 32
    # the remainder of 33 is 32, itself one chunk
    assert first[33 - first[33]] == 32


def test_extra_chunk_is_charged():
    rate = {n: 1.0 for n in range(1, 65)}
    rate[32] = 1.01  # 1% faster: less than the 2% charge of an extra chunk
    first = first_chunks(rate)
    assert first[33] == 33
