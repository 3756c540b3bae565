"""Helpers to read the C ABI declared under include/ (used by the ABI tests)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header: str = "wxpy.h") -> list[str]:
    """Names of the functions declared in include/<header> (comments stripped)."""
    names = []
    for path in [os.path.join(ROOT, "include", header)]:
        with open(path) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        src = re.sub(r"#[^\n]*", " ", src)
        for m in re.finditer(r"\b(wxpy\w*)\s*\(", src):
            names.append(m.group(1))
    return sorted(set(names))
