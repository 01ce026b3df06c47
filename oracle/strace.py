"""strace text -> event table, the front end of the paper's monitor (Sec. 5:
a parsing module translates strace strings into a numerical table).  Test
infrastructure only.

A line reads  [pid] TIME NAME(ARGS...) = RET [ERRNO (text)]  where the pid
is "[pid N]" or a number followed by blanks, and TIME is seconds.fraction
(strace -ttt) or HH:MM:SS.fraction (-tt), the fraction read as microseconds.
A line whose NAME has a rule becomes an event (key, code, microseconds):
the key is the first argument or the return value, as the rule says.  strace
-f splits a call into "NAME(ARGS <unfinished ...>" and "<... NAME resumed>
...) = RET"; the half that holds the key gives the event.  Lines of other
calls, signals and exits, lines without their key, calls returning a
negative value when the rule asks for success, and return-value keys that
are negative are dropped.
"""
from __future__ import annotations

import re
from dataclasses import dataclass

ARG0, RET = 0, 1


@dataclass
class Rule:
    name: str
    code: int
    key_from: int      # ARG0 or RET
    ok_only: bool = False


_PID_BRACKET = re.compile(r"\[pid\s+(\d+)\]\s*")
_PID_PLAIN = re.compile(r"(\d+)[ \t]+")
_TIME = re.compile(r"(\d+):(\d+):(\d+)(?:\.(\d+))?|(\d+)(?:\.(\d+))?")
_NAME = re.compile(r"[A-Za-z0-9_]+")
_INT = re.compile(r"-?(?:0[xX][0-9A-Fa-f]+|\d+)")


def _micro(frac):
    if not frac:
        return 0
    return int((frac + "000000")[:6])


def _int(s):
    m = _INT.match(s)
    if not m:
        return None
    t = m.group(0)
    neg = t.startswith("-")
    t = t.lstrip("-")
    v = int(t, 16) if t[:2].lower() == "0x" else int(t)
    return -v if neg else v


def parse_line(line: str, rules: dict):
    """(key, code, microseconds) of one line, or None if it is dropped."""
    s = line.rstrip("\r").lstrip(" \t")
    m = _PID_BRACKET.match(s) if s.startswith("[pid") else _PID_PLAIN.match(s)
    if s.startswith("[pid") and not m:
        return None
    if m:
        s = s[m.end():]
    m = _TIME.match(s)
    if not m or not m.group(0):
        return None
    if m.group(1) is not None:
        secs = int(m.group(1)) * 3600 + int(m.group(2)) * 60 + int(m.group(3))
        us = _micro(m.group(4))
    else:
        secs, us = int(m.group(5)), _micro(m.group(6))
    s = s[m.end():].lstrip(" \t")
    resumed = s.startswith("<... ")
    if resumed:
        s = s[5:]
    m = _NAME.match(s)
    if not m or m.group(0) not in rules:
        return None
    rule = rules[m.group(0)]
    rest = s[m.end():]
    if resumed:
        if not rest.startswith(" resumed>"):
            return None
        rest = rest[len(" resumed>"):]
    elif not rest.startswith("("):
        return None
    else:
        rest = rest[1:]
    unfinished = line.rstrip("\r").endswith("<unfinished ...>")
    ret = None
    if not unfinished:
        k = rest.rfind(") = ")
        if k >= 0:
            ret = _int(rest[k + 4:].lstrip(" \t"))
    if rule.key_from == ARG0:
        if resumed:
            return None
        key = _int(rest.lstrip(" \t"))
        if key is None or key < 0:
            return None
        if rule.ok_only and ret is not None and ret < 0:
            return None
    else:
        if ret is None or ret < 0:
            return None
        key = ret
    return key, rule.code, secs * 1_000_000 + us


def parse(text: str, rules):
    """Event table of a whole log: lists keys, codes, microseconds in line order."""
    table = {r.name: r for r in rules}
    lines = text.split("\n")
    if lines and lines[-1] == "":
        lines.pop()
    keys, codes, ts = [], [], []
    for line in lines:
        e = parse_line(line, table)
        if e is not None:
            keys.append(e[0])
            codes.append(e[1])
            ts.append(e[2])
    return keys, codes, ts
