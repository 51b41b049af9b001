"""Write input_digests.txt: SHA-256 digests of a few generated instances'
arrays.  Calls only the seeded generator (no solver arithmetic)."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_2206_03203_gb300 import inputs  # noqa: E402


def digests():
    i = inputs.random_segments_2d(contrast=1e4)
    b = inputs.batch_instance(5)
    return {"seg2d_1024_c1e4_km": hashlib.sha256(i.km.tobytes()).hexdigest(),
            "seg2d_1024_c1e4_kf": hashlib.sha256(i.fc_kf.tobytes()).hexdigest(),
            "batch3d_256_i5_km_kf_pD": hashlib.sha256(b.km.tobytes() + b.fc_kf.tobytes() +
                                                      b.pD_left.tobytes()).hexdigest()}


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "input_digests.txt")
    head = open(out).read().split("\n")[:3] if os.path.exists(out) else []
    lines = [l for l in head if l.startswith("#")] + [f"{k} {v}" for k, v in digests().items()]
    open(out, "w").write("\n".join(lines) + "\n")
