"""The log-odds oracle against its pins, and planted mistakes in copies of it
(CPU only; the committed oracle is never modified)."""
import os
import types

import pytest

import oracle
import oracle.logodds
from logodds_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "logodds.py")

# (name, text in logodds.py, replacement)
MUTANTS = [
    ("dropped prior term", "return (log_post + log_prior_bar) - (log_post_bar + log_prior)",
     "return log_post - log_post_bar"),
    ("complement includes the class", "logsumexp(np.delete(L, c, axis=1), axis=1)", "logsumexp(L, axis=1)"),
    ("sign of the kernel", "L = -float(beta) * D", "L = float(beta) * D"),
    ("prior odds of one", "log_prior_bar = np.log((n_cls - 1) / n_cls)", "log_prior_bar = np.log(1.0 / n_cls)"),
    ("kernel with beta / 2", "L = -float(beta) * D", "L = -0.5 * float(beta) * D"),
    ("zero increments counted as positive", "use = rows > 0 if", "use = rows >= 0 if"),
    ("positive-only ignored", "use = rows > 0 if positive_only else np.ones(rows.shape, bool)",
     "use = np.ones(rows.shape, bool)"),
    ("argmax ties to the highest class", "classes = np.argmax(totals, axis=1)",
     "classes = totals.shape[1] - 1 - np.argmax(totals[:, ::-1], axis=1)"),
    ("argmin instead of argmax", "classes = np.argmax(totals, axis=1)", "classes = np.argmin(totals, axis=1)"),
    ("image rows off by one", "rows = inc[offsets[g]:offsets[g + 1]]", "rows = inc[offsets[g]:offsets[g + 1] + 1]"),
]


def _mutant(text, repl):
    with open(SRC) as f:
        src = f.read()
    assert src.count(text) >= 1, text
    mod = types.ModuleType("logodds_mutant")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(text, repl), "logodds_mutant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    pin(oracle.logodds)


@pytest.mark.parametrize("name,text,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, text, repl):
    mod = _mutant(text, repl)
    failed = []
    for pin in ALL_PINS:
        try:
            pin(mod)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin catches the mutant '{name}'"


def test_rejects_one_class():
    import numpy as np
    with pytest.raises(ValueError):
        oracle.logodds.logodds_increments(np.zeros((3, 1), np.int64), 1.0)
