"""Autotuner placeholder: cache location and loader (the tuner itself lands next)."""
import json
import os


def cache_path():
    return os.environ.get("COFFEE_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                            "tune_cache.json"))


def load_cache():
    p = cache_path()
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        return json.load(f).get("entries", {})
