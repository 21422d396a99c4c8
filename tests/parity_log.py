"""Record of the measured errors of the CUDA path against the FP64 oracle.

Test infrastructure.  When the environment variable OPO_PARITY_LOG names a
file, every parity comparison that calls :func:`record` appends one JSON line
to it (test, case, precision, path, worst relative L2 error over the fields
and over the output fields, worst relative error of the output powers, and the
centroid error in units of the spectral width).  Without the variable nothing
is written.  The tables of measured errors are built from these lines.
"""
import json
import os

PREC_NAMES = {0: "fp64", 1: "fp32+ph64"}
PATH_NAMES = {0: "auto", 1: "plain", 2: "fused"}


def record(test, case, precision, path, **values):
    fn = os.environ.get("OPO_PARITY_LOG")
    if not fn:
        return
    row = {"test": test, "case": case, "precision": PREC_NAMES.get(precision, precision),
           "path": PATH_NAMES.get(path, path)}
    row.update({k: (float(v) if isinstance(v, (int, float)) else v) for k, v in values.items()})
    with open(fn, "a") as fh:
        fh.write(json.dumps(row) + "\n")
