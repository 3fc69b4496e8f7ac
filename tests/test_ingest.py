"""Edge-list files (Section II's inputs) read by the library's host reader:
tab-separated 1-based "u v weight" lines and Matrix Market coordinate files,
ids made 0-based, weights ignored, comments skipped, malformed input
reported.  Host code only: these run without a GPU."""
import numpy as np
import pytest

import paper_1708_06866_gb300 as tc


def write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_tab_separated_with_weights_and_comments(tmp_path):
    # Fig. 1's diamond as the Graph Challenge writes it: both directions, weight 1
    text = "# diamond\n1\t2\t1\n2\t1\t1\n1\t3\t1\n3\t1\t1\n\n2\t3\t1\n3\t2\t1\n" \
           "2\t4\t1\n4\t2\t1\n3\t4\t1\n4\t3\t1\n"
    src, dst, n = tc.tc_read_edges(write(tmp_path, "fig1.tsv", text))
    assert n == 4 and len(src) == 10
    assert src.tolist() == [0, 1, 0, 2, 1, 2, 1, 3, 2, 3]
    assert dst.tolist() == [1, 0, 2, 0, 2, 1, 3, 1, 3, 2]


def test_spaces_no_trailing_newline_and_loops_are_kept(tmp_path):
    src, dst, n = tc.tc_read_edges(write(tmp_path, "g.txt", "5 5\n1 7 0.5\n7 1"))
    assert n == 7
    assert src.tolist() == [4, 0, 6] and dst.tolist() == [4, 6, 0]


def test_matrix_market_pattern_and_values(tmp_path):
    text = ("%%MatrixMarket matrix coordinate pattern symmetric\n% a comment\n"
            "6 6 3\n2 1\n3 1\n6 5\n")
    src, dst, n = tc.tc_read_edges(write(tmp_path, "a.mtx", text))
    assert n == 6 and src.tolist() == [1, 2, 5] and dst.tolist() == [0, 0, 4]
    text = "%%MatrixMarket matrix coordinate real general\n3 4 2\n1 4 2.5\n3 2 -1e3\n"
    src, dst, n = tc.tc_read_edges(write(tmp_path, "b.mm", text))
    assert n == 4 and src.tolist() == [0, 2] and dst.tolist() == [3, 1]
    # format forced regardless of the name
    src2, dst2, n2 = tc.tc_read_edges(write(tmp_path, "b.dat", text), fmt=2)
    assert src2.tolist() == [0, 2] and n2 == 4


def test_empty_file(tmp_path):
    src, dst, n = tc.tc_read_edges(write(tmp_path, "e.tsv", "# nothing\n\n"))
    assert len(src) == 0 and n == 0


@pytest.mark.parametrize("name,text,code", [
    ("z.tsv", "0\t1\t1\n", tc.TC_ERANGE),                       # ids are 1-based
    ("big.tsv", "1\t2147483648\t1\n", tc.TC_ERANGE),            # above 2^31 - 1
    ("bad.tsv", "1\tx\t1\n", tc.TC_EINVAL),
    ("one.tsv", "1\n", tc.TC_EINVAL),
    ("neg.tsv", "-1\t2\n", tc.TC_EINVAL),
    ("h.mtx", "%%MatrixMarket matrix array real general\n2 2\n1\n", tc.TC_EINVAL),
    ("n.mtx", "%%MatrixMarket matrix coordinate pattern general\n3 3 2\n1 2\n", tc.TC_EINVAL),
    ("o.mtx", "%%MatrixMarket matrix coordinate pattern general\n3 3 1\n1 4\n", tc.TC_ERANGE),
    ("x.mtx", "not a header\n1 2\n", tc.TC_EINVAL),
])
def test_malformed_inputs_are_reported(tmp_path, name, text, code):
    with pytest.raises(tc.TCError) as ei:
        tc.tc_read_edges(write(tmp_path, name, text))
    assert ei.value.code == code


def test_missing_file_and_small_capacity(tmp_path):
    with pytest.raises(tc.TCError):
        tc.tc_read_edges(str(tmp_path / "missing.tsv"))
    lib = tc.load_library()
    import ctypes
    path = write(tmp_path, "c.tsv", "1\t2\n2\t3\n").encode()
    src = np.empty(1, dtype=np.int32)
    dst = np.empty(1, dtype=np.int32)
    m, n = ctypes.c_int64(), ctypes.c_int32()
    rc = lib.tc_read_edges(path, 0, src.ctypes.data, dst.ctypes.data, 1, ctypes.byref(m),
                           ctypes.byref(n))
    assert rc == tc.TC_EINVAL and m.value == 2


def test_long_lines(tmp_path):
    text = "1\t2\t" + "9" * 200000 + "\n2\t3\t1\n"
    src, dst, n = tc.tc_read_edges(write(tmp_path, "long.tsv", text))
    assert src.tolist() == [0, 1] and dst.tolist() == [1, 2] and n == 3
