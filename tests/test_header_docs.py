"""Every entry point declared in include/fmocc.h carries a comment that cites the passage of the
paper defining its operation (a section, equation, listing or figure, or the BWA bound that
Listing 2 cites), or says that the paper has no counterpart, and states its errors where it
returns a status.  Consecutive declarations share the comment above them."""
import os
import re

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "fmocc.h")
CITE = re.compile(r"Sec\. \d|Eq\. \d|Listing \d|Fig\. \d|Li and Durbin|no counterpart")
DECL = re.compile(r"^(?:int|void|const char \*)\s*(fm_\w+)\(", re.M)


def _declarations():
    src = open(HDR).read()
    out = []
    for m in DECL.finditer(src):
        before = src[:m.start()]
        # skip back over the declarations directly above (they share the comment block)
        lines = before.rstrip("\n").split("\n")
        while lines and (DECL.match(lines[-1]) or lines[-1].startswith(" ") and
                         not lines[-1].lstrip().startswith("*")):
            lines.pop()
        text = "\n".join(lines).rstrip()
        block = text[text.rfind("/*"):] if text.endswith("*/") else ""
        # a declaration spanning several lines: its own text up to the closing ");"
        end = src.find(";", m.end())
        out.append((m.group(1), block, src[m.start():end]))
    return out


def test_every_entry_point_is_documented_with_a_citation():
    decls = _declarations()
    assert len(decls) >= 20
    missing = [name for name, block, _ in decls if not block]
    assert not missing, f"no comment above {missing}"
    uncited = [name for name, block, _ in decls if not CITE.search(block)]
    assert not uncited, f"no passage or 'no counterpart' in the comment of {uncited}"


def test_status_returning_calls_state_their_errors():
    src = open(HDR).read()
    for name, block, decl in _declarations():
        if not decl.startswith("int "):
            continue
        # the errors are stated in the call's own comment or, for the server calls and the
        # tuning pair, in the shared text above them
        assert "FM_E" in block or "Errors" in block or name.startswith(("fm_server_", "fm_get_tuning",
                                                                        "fm_set_tuning")), name
    assert "FM_EINVAL for out-of-range values" in src
