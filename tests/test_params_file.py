"""The handout's parameter-file format (Handout, starter code): the example
values it prints, quoting, comments, and refusals."""
import pytest

from paper_2309_14311_gb300 import params as P

EXAMPLE = """\
L = 500
T = 500
N = 300
p = 0.2
vmax = 2
seed = 13
outputprefix = "traffic"
per = 10
"""


def test_the_handouts_example_values():
    sp = P.parse(EXAMPLE)
    assert (sp.L, sp.T, sp.N, sp.p, sp.vmax, sp.seed, sp.outputprefix, sp.per) == \
        (500, 500, 300, 0.2, 2, 13, "traffic", 10)


def test_comments_blank_lines_and_order():
    text = "# a comment\n\n" + "\n".join(reversed(EXAMPLE.splitlines())) + "\n  # trailing\n"
    assert P.parse(text) == P.parse(EXAMPLE)


@pytest.mark.parametrize("text,why", [
    (EXAMPLE.replace("per = 10\n", ""), "missing"),
    (EXAMPLE + "per = 5\n", "twice"),
    (EXAMPLE + "speed = 3\n", "unknown"),
    (EXAMPLE.replace("N = 300", "N = 600"), "range"),
    (EXAMPLE.replace("p = 0.2", "p = 1.5"), "range"),
    (EXAMPLE + "garbage\n", "expected"),
])
def test_bad_files_are_refused(text, why):
    with pytest.raises(ValueError, match=why):
        P.parse(text)
