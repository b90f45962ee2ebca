import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    # temporary paths of the tests live in the repository's git-ignored
    # build folder (pytest empties it at the start of a session)
    if not config.option.basetemp:
        os.makedirs(os.path.join(ROOT, "_build"), exist_ok=True)
        config.option.basetemp = os.path.join(ROOT, "_build", "pytest_tmp")
    if not hasattr(config, "workerinput"):  # the build artefacts of the last session
        import shutil
        shutil.rmtree(os.path.join(ROOT, "_build", "tmp"), ignore_errors=True)
