"""B300-native engine for the process-mining summaries of PM4Py-GPU
(arXiv 2204.04898): formatting a columnar event log by (case, timestamp, row),
the frequency and performance directly-follows graphs, start/end activities,
variants and drill-down filters.

The compute path is the CUDA library libpm4g.so (C ABI in include/pm4g.h);
``paper_2204_04898_b300.pm4g`` binds it with the same function names.
"""

import os as _os

# where build.py writes the library (not imported from it, so that
# ``python -m paper_2204_04898_b300.build`` runs the module only once)
LIBRARY_PATH = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "libpm4g.so")
