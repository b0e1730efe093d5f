"""The in-tree build (no GPU needed): every translation unit compiles for
sm_103a and links, and the library is relinked whenever it is older than one
of its objects, so a link that failed after compiling never leaves an older
library in use."""
import os

from paper_2604_02125_gb300 import build


def test_library_relinked_when_older_than_an_object():
    lib = build.build()
    objs = sorted(os.path.join(build.BUILD, f) for f in os.listdir(build.BUILD) if f.endswith(".o"))
    assert objs and os.path.exists(lib)
    before = os.path.getmtime(lib)
    # an object newer than the library, as after a link that failed
    os.utime(objs[0], (before + 2, before + 2))
    os.utime(lib, (before, before))
    build.build()
    assert os.path.getmtime(lib) > before
