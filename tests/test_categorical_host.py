"""Categorical front end (Sec. 1, "Extension for categorical data
compression"), no GPU: the oracle's encoding against the definition, the
factor-2 identity between the one-hot Hamming distance and the categorical
distance, and the host-side label encoding."""
import numpy as np

import oracle
from paper_1910_04658_gb300 import categorical


def test_onehot_matches_dense_definition():
    cards = [3, 1, 5, 2]
    labels = np.array([[0, 0, 4, 1], [2, 0, 0, 0], [1, 0, 3, 1]])
    rp, col, d = oracle.onehot(labels, cards)
    assert d == 11 and rp.tolist() == [0, 4, 8, 12]
    dense = np.zeros((3, d), np.int64)
    for i in range(3):
        dense[i, col[rp[i]:rp[i + 1]]] = 1
    expect = np.zeros((3, d), np.int64)
    base = np.cumsum([0] + cards[:-1])
    for i in range(3):
        for f in range(4):
            expect[i, base[f] + labels[i, f]] = 1
    assert np.array_equal(dense, expect)
    assert categorical.feature_offsets(cards).tolist() == [0, 3, 4, 9, 11]


def test_hamming_of_onehot_is_twice_the_categorical_distance():
    # the paper states equality; each differing feature flips two bits
    cards = [4, 7, 2, 30, 3, 11]
    lab = categorical.synthetic(5, 120, cards)
    rp, col, d = oracle.onehot(lab, cards)
    pa, pb = np.triu_indices(120, 1)
    ham = oracle.exact_pairs(rp, col, pa, pb)[:, 1]
    dist = np.array([oracle.categorical_distance(lab[a], lab[b]) for a, b in zip(pa, pb)])
    assert np.array_equal(ham, 2 * dist)
    assert (dist > 0).any() and (dist == 0).any()


def test_label_encode_roundtrip():
    cols = [["rain", "sun", "sun", "fog"], [3, 1, 3, 2], [0.5, 0.5, 0.5, 0.5]]
    labels, classes = categorical.label_encode(cols)
    assert labels.shape == (4, 3) and labels.dtype == np.uint32
    assert labels[:, 0].tolist() == [1, 2, 2, 0]            # sorted classes: fog, rain, sun
    for f, c in enumerate(cols):
        assert list(classes[f][labels[:, f]]) == list(c)
        assert labels[:, f].max() < len(classes[f])


def test_synthetic_labels_in_range():
    cards = [2, 10, 100]
    lab = categorical.synthetic(1, 500, cards)
    assert lab.shape == (500, 3)
    for f, m in enumerate(cards):
        assert lab[:, f].max() < m
