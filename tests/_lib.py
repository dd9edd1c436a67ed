"""Shared test helpers: build the library once per session and load it."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mfipm.h")


def header_functions():
    """Names of the functions declared in include/mfipm.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mfipm_\w+)\s*\(", src)))


def built_lib():
    from paper_1208_5435_gb300 import build
    build.build()
    from paper_1208_5435_gb300 import _capi
    return _capi.lib()
