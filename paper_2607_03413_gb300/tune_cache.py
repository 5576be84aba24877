"""Autotuned kernel variants kept across runs in a JSON file.

The autotuners of the library (cw_op_autotune, cw_batch_autotune) time every kernel variant on the
device; their choice depends on the GPU, the operator (degree, kind, geometry mode, precision) and the
size of the work, not on the vector values. A cache keyed by exactly these lets a later run set the
chosen variant without timing again. The file is rewritten atomically (temporary file + rename), so a
reader never sees a partial file; an unreadable or foreign file is ignored and replaced.
"""
import json
import os

_VERSION = 1


class TuneCache:
    def __init__(self, path):
        self.path = path
        self.entries = {}
        try:
            with open(path) as f:
                data = json.load(f)
            if isinstance(data, dict) and data.get("version") == _VERSION and isinstance(data.get("entries"), dict):
                self.entries = data["entries"]
        except (OSError, ValueError):
            pass

    @staticmethod
    def key(*parts):
        return "|".join(str(p) for p in parts)

    def get(self, key):
        return self.entries.get(key)

    def put(self, key, value):
        self.entries[key] = value
        self.save()

    def save(self):
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump({"version": _VERSION, "entries": self.entries}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def device_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())
