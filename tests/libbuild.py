"""Build-once helper for the tests (the library is built in-tree)."""
import os
import threading

_lock = threading.Lock()
_done = False


def ensure_built():
    global _done
    with _lock:
        if not _done:
            from paper_2003_02450_gb300 import build
            build.build()
            _done = True
