"""Every entry point declared in include/jslam.h states, in the comment
above its declaration, the passage of the paper that defines the operation
(a section or an equation) or that the paper has no counterpart for it."""
import os
import re

from conftest import ROOT

# The calls of the boundary table of the hot path; each must be declared.
BOUNDARY = ("jslam_create", "jslam_extract", "jslam_extract_batch", "jslam_match", "jslam_get_keypoints",
            "jslam_sync", "jslam_set_skip_model", "jslam_destroy", "jslam_status_str")

CITATION = re.compile(r"Sec\.\s+(?:II|III|IV|V)(?:-[A-H](?:-\d)?)?|Eq\.\s+\d|no counterpart in the paper", re.I)


def _units():
    """(name, text before the declaration back to the previous declaration)."""
    text = open(os.path.join(ROOT, "include", "jslam.h")).read()
    text = text[text.index("extern \"C\" {"):]
    units, prev = [], 0
    for m in re.finditer(r"^(?:[a-z_][\w ]*?[\s*]+)(jslam_[a-z_]+)\s*\([^;{]*?\)\s*;", text, flags=re.M | re.S):
        units.append((m.group(1), text[prev:m.start()]))
        prev = m.end()
    return units


def test_every_declaration_has_a_unit():
    names = [n for n, _ in _units()]
    assert len(names) == len(set(names))
    from test_abi import _declared_functions
    assert sorted(names) == _declared_functions()
    for call in BOUNDARY:
        assert call in names, call


def test_every_entry_point_cites_its_passage():
    missing = []
    for name, before in _units():
        comments = " ".join(re.findall(r"/\*.*?\*/", before, flags=re.S))
        comments = re.sub(r"\s*\n\s*\*\s?", " ", comments)  # join the comment's lines
        if not CITATION.search(comments):
            missing.append(name)
    assert not missing, f"no passage cited for: {missing}"


def test_citation_pattern_rejects_plain_prose():
    assert not CITATION.search("/* Release the context and everything it owns. */")
    assert CITATION.search("Sec. II-C-2") and CITATION.search("Eq. 3") and CITATION.search("no counterpart in the paper")
