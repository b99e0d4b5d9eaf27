"""The register sorting network of the extraction fill's lane path (8 keys): the
comparator table is read from the kernel source and applied to all 256 0/1 inputs;
by the 0-1 principle a comparator network that sorts every 0/1 sequence sorts every
sequence.  A network with a dropped or misplaced comparator fails here."""
import itertools
import os
import re

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2509_20776_gb300", "csrc", "extract_rows.cuh")


def network():
    text = open(SRC).read()
    m = re.search(r"void sort8\(.*?constexpr int P\[(\d+)\]\[2\] = \{(.*?)\};", text, re.S)
    assert m, "sort8's comparator table not found"
    pairs = [(int(a), int(b)) for a, b in re.findall(r"\{(\d+),\s*(\d+)\}", m.group(2))]
    assert len(pairs) == int(m.group(1))
    return pairs


def apply(net, xs):
    xs = list(xs)
    for a, b in net:
        assert 0 <= a < b < 8
        if xs[b] < xs[a]:
            xs[a], xs[b] = xs[b], xs[a]
    return xs


def test_sort8_sorts_every_01_input():
    net = network()
    for bits in itertools.product((0, 1), repeat=8):
        assert apply(net, bits) == sorted(bits), bits


def test_sort8_moves_values_with_keys():
    net = network()
    keys = [7, 3, 0xFFFFFFFF, 5, 0, 0xFFFFFFFF, 2, 9]
    pairs = apply(net, [(k, i) for i, k in enumerate(keys)])
    assert [k for k, _ in pairs] == sorted(keys)
    assert all(keys[i] == k for k, i in pairs)


def test_sort8_would_catch_a_missing_comparator():
    net = network()
    for drop in range(len(net)):
        broken = net[:drop] + net[drop + 1:]
        assert any(apply(broken, b) != sorted(b) for b in itertools.product((0, 1), repeat=8)), drop
